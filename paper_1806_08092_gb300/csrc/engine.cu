// Per-iteration scatter/gather engine (Alg. 2 with Alg. 3 and Eq. (mode)).
//
// One iteration = up to six launches on the caller's stream, after the host has read the plan:
//   k_plan        1 CTA: per-partition V_a/E_a from the previous gather, mode
//                 choice (Eq. (mode), forced, or learned), PC/NULL actions,
//                 SC work list, termination test (Sec. 3.1.x active lists); its
//                 control snapshot goes straight to mapped host memory.
//   k_scatter_pc  PC mode (Alg. 3): every PNG slot of a PC partition receives
//                 the current value of its source (NULL if inactive) as a
//                 sequential vectorised stream over the padded row.
//   k_scatter_sc  SC mode (Alg. 2 scatter): active vertices of the partition
//                 append (destination, value) pairs to their bins through
//                 warp-aggregated cursors.
//   k_gather_pc   PC part of the gather: each column's bins staged block by
//                 block in shared memory by bulk copies, folded through the
//                 destination-sorted entry lists into a shared accumulator
//                 (lane-serial runs and segmented warp scans, no atomics).
//   k_merge_pc    columns split over several PC gather tasks: partial vectors
//                 combined in task order.
//   k_gather      per (column q, destination range) task: the column's PC
//                 result and the task's SC pairs, then reInit/gather/filter user
//                 functions and the next frontier (Alg. 2 gather + filter; Sec. 4).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "gpop_internal.cuh"

namespace gpop {

// ALG_MSBFS: BFS from up to 32 sources at once (gpop_run_msbfs); a vertex's state is the set of sources
// that reached it and its message the complement of the sources it reached in the last iteration
enum Algo : int {
    ALG_PR = GPOP_PAGERANK, ALG_BFS = GPOP_BFS, ALG_CC = GPOP_CC, ALG_SSSP = GPOP_SSSP, ALG_PPR = GPOP_PPR,
    ALG_NIBBLE = GPOP_NIBBLE, ALG_MSBFS = 6
};
// applications whose messages are FP32 values combined by addition
__host__ __device__ constexpr bool sums(int a) { return a == ALG_PR || a == ALG_PPR || a == ALG_NIBBLE; }

constexpr int kGatherThreads = 256;
constexpr int kGatherWarps = kGatherThreads / 32;
constexpr int kScatterThreads = 256;    // k_scatter_sc
constexpr int kScatterPcThreads = 512;  // k_scatter_pc
constexpr int kPlanThreads = 1024;
constexpr uint32_t kPlanLoads = 3;  // gather-task statistics a plan thread loads at once
// The L1 change of a gather task (at most 2: a change of probability mass) is passed to the plan as an
// unsigned fixed-point number with 62 fraction bits, so that the plan sums it exactly, in any order,
// with integer adds (FP64 arithmetic is scarce on this GPU); the rounding is below 2^-62 per task.
constexpr double kResOne = 0x1p62, kResUnit = 0x1p-62;
constexpr uint32_t kSent = 0xFFFFFFFFu;
constexpr uint32_t kScUnitEdges = 1u << 12;  // active edges per SC scatter unit (a partition with more is split)
constexpr uint32_t kScSegs = 16;              // 1024-vertex segments per partition (P <= 16384)
constexpr uint32_t kBigScBin = 2048;     // SC bins at least this large are folded by the whole gather CTA
constexpr uint32_t kMaxBigScBins = 64;
constexpr int kPcWarps = kPcGatherWarps;          // k_gather_pc consumer warps (one destination slice of a block each)
constexpr int kPcThreads = 32 * (kPcWarps + 1);   // + the producer warp
constexpr uint32_t kPcMaxBufs = 4;                // value buffers of k_gather_pc (blocks staged ahead)
constexpr uint32_t kPcSpinLimit = 1u << 24;       // tries of a bounded mbarrier wait
constexpr unsigned long long kPcWaitNs = 2000000000ull;  // ... and its time limit (2 s)
constexpr uint32_t kPcSleepNs = 20000;            // k_gather_pc: a waiting warp sleeps up to 20 us per try
static_assert(kPcRound == 32 * 16, "a full round gives each lane 16 entries");

struct Params {
    // graph
    uint32_t V, P, shift, k;
    const uint32_t *rowptr, *col;
    const int32_t *w;
    const uint16_t *esub;
    const uint32_t *row_bin, *bin_q, *col_bin, *col_bins;
    const uint32_t *sub_cap, *sub_task, *row_sub, *task_sub_ptr;
    const uint16_t *png;
    uint32_t *pdata;
    const uint32_t *row_png;
    uint2 *scpair;
    uint32_t *sccnt;
    uint32_t *task_sc_cnt, *task_sc_list;  // per gather task: fresh SC bins of this iteration
    // PC gather blocks
    const uint4 *pc_runs, *pc_task;
    const uint32_t *pc_wsp, *pc_tsp;  // per task block: kPcWarps+1 entry splits; per task: first split row
    const uint2 *pc_blk_prange;       // per block: first and last source partition of its bins
    uint32_t *pc_prefix;              // per iteration: PC partitions before p (k+1 entries)
    const uint32_t *pc_blk_run, *pc_blk_nval, *pc_blk_ent, *col_ntask, *col_part0, *pe;
    const int32_t *pw;
    uint32_t *pc_part;
    uint32_t npct;
    const uint2 *pc_merge;  // merge items of split columns
    uint32_t nmerge;
    uint32_t pc_nbuf;   // value buffers of k_gather_pc (2..kPcMaxBufs)
    uint32_t *pc_sum;  // per vertex: combined PC message of the iteration (single-task columns)
    const uint32_t *Ep, *npng_p;
    const GatherTask *gtask;
    uint32_t ngt;
    const uint32_t *col_task;
    const ScatterTask *stask;
    uint32_t nst;
    uint8_t *pc_state;
    // run state
    uint32_t *val, *lvl, *sval, *bits;
    uint32_t *t_va;
    unsigned long long *t_ea;
    unsigned long long *t_res;  // L1 change of each gather task: fixed point, kResOne = 1
    uint32_t *t_stamp;
    uint8_t *mode, *action;
    uint32_t *gflag, *gflag_pc, *counters;
    uint4 *sc_list;                   // SC scatter units: (partition, unit, units, active edges)
    uint32_t *sc_seg;                 // active out-edges of each 1024-vertex segment of the SC partitions [k][16]
    uint32_t *sc_gcur, *sc_udone;     // split SC partitions: bin cursors and finished units (zero at rest)
    Control *ctrl;
    Control *ctrl_snap;     // the plan's snapshot for the host: mapped pinned memory, slot (iter - 1) & 1
    const float *selector;  // learned selector parameters (W1, W2 transposed) or null
    uint8_t *sel_mode;      // learned policy: per-partition choice for the next plan (k_select / k_gather tail)
    uint32_t *col_done;     // learned policy: finished gather tasks per column (zero at rest)
    uint32_t pc_skip;       // k_gather_pc: skip blocks without PC sources (some partition is not PC)
    // work lists / timing used by the SC scatter and by the LOG_BOTH shadow launches
    const uint4 *list;           // units for k_scatter_sc
    const uint32_t *list_count;  // number of entries in list
    uint32_t counter_slot;       // which counters[] entry the launch consumes
    uint32_t dry;                // shadow launch: do not publish bins or flags
    unsigned long long *t_task;  // per-task CTA durations (ns) or null
    unsigned long long *t_gpc;   // LOG_BOTH: CTA time of k_gather_pc (ns, all CTAs) or null
    unsigned long long *t_gsc;   // LOG_BOTH: CTA time of k_gather's SC passes (ns) or null
    unsigned long long *gath;    // destinations visited by k_gather over the run
    uint4 *all_list;             // LOG_BOTH: units of every partition scattered this iteration
    float *feat;                 // LOG_BOTH: per-partition selector features [k][8]
    uint32_t *part_va;           // LOG_BOTH: V_a per partition
    unsigned long long *part_ea; // LOG_BOTH: E_a per partition
    uint32_t log_both;
    // per launch
    uint32_t epoch, iter, source, max_iters;
    const uint32_t *msrc;   // multi-source BFS: the pass's sources (nsrc <= 32; bit j of a set = msrc[j])
    uint32_t nsrc;
    uint32_t *lvl_ms;       // multi-source BFS: levels, row j (V words) for source msrc[j]
    float c0, c1;           // PR: (1-d)/V, d.  PPR: alpha, 1-alpha
    float eps;              // Nibble: the threshold per unit of out-degree
    double t_res0;          // resumed run: the L1 change of the last gather before the state was saved
    double tol;
    int algo, policy;
    uint32_t bw_num, bw_den;
    uint32_t isg_w;         // interleaved scatter-gather: waves (0: off)
};

// --- small device helpers ----------------------------------------------------------------------

__device__ __forceinline__ float u2f(uint32_t x) { return __uint_as_float(x); }
__device__ __forceinline__ uint32_t f2u(float x) { return __float_as_uint(x); }
// BF16 message bins (PR / PPR with msg_bf16): a message value rounds to BF16 (nearest even) on its way into
// a bin and widens back to FP32 in the gather; NULL is 0xFFFF (a NaN no rounding produces from the
// non-negative values these applications send)
constexpr uint32_t kNull16 = 0xFFFFu;
__device__ __forceinline__ uint32_t to_bf16(uint32_t x) {
    return x == kNull ? kNull16 : (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(__uint_as_float(x)));
}
__device__ __forceinline__ uint32_t from_bf16(uint32_t h) { return h << 16; }  // FP32 bits of a BF16 value

template <int ALGO>
struct Op {
    // monoid used to combine the messages a vertex receives in one gather: FP32 sum (PR / PPR), minimum
    // (BFS parent, CC label, SSSP distance) or bitwise AND (multi-source BFS: messages are complemented
    // source sets, so the AND is the complement of their union).  Except for the sums the identity is
    // 0xFFFFFFFF, the NULL of an inactive source, which therefore folds as a no-op.
    static __device__ __forceinline__ uint32_t identity() {
        return sums(ALGO) ? 0u : kInf;
    }
    static __device__ __forceinline__ uint32_t combine(uint32_t a, uint32_t b) {
        if (sums(ALGO)) return f2u(u2f(a) + u2f(b));
        if (ALGO == ALG_MSBFS) return a & b;
        return a < b ? a : b;
    }
    // applyWeight of Alg. 7 (SSSP adds the edge weight, saturating below kInf)
    static __device__ __forceinline__ uint32_t weigh(uint32_t x, int32_t w) {
        if (ALGO == ALG_SSSP) {
            uint64_t s = (uint64_t)x + (uint32_t)w;
            return s >= kInf ? kInf - 1 : (uint32_t)s;
        }
        return x;
    }
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive scan across a block of blockDim.x threads (multiple of 32, <= 1024)
__device__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_warp, uint32_t *total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(x, lane);
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < nw ? s_warp[lane] : 0;
        uint32_t ti = warp_incl_scan(t, lane);
        if (lane < nw) s_warp[lane] = ti - t;
        if (lane == nw - 1) s_warp[32] = ti;
    }
    __syncthreads();
    uint32_t r = inc - x + s_warp[wid];
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

// Work units of one chunk of partitions, written by every thread of the block: thread t has cnt units,
// the first at position beg (an exclusive scan over the chunk, tot units in all), for partition q with ea
// active edges.  A hub partition can have thousands of units, so instead of its partition's thread writing
// them all, the block's threads take equal ranges of consecutive units: a binary search over the chunk's
// unit ends finds the partition of a range's first unit, and the rest follow by walking forward.
__device__ void write_units(uint4 *list, uint32_t base, uint32_t q, uint32_t cnt, uint32_t beg, uint32_t tot, uint32_t ea,
                            uint32_t *s_beg, uint32_t *s_end, uint32_t *s_q, uint32_t *s_ea) {
    s_beg[threadIdx.x] = beg;
    s_end[threadIdx.x] = beg + cnt;
    s_q[threadIdx.x] = q;
    s_ea[threadIdx.x] = ea;
    __syncthreads();
    const uint32_t per = (tot + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = threadIdx.x * per, i1 = min(tot, i0 + per);
    if (i0 < i1) {
        uint32_t lo = 0, hi = blockDim.x - 1;  // first thread whose units end after i0
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_end[mid] > i0) hi = mid; else lo = mid + 1;
        }
        for (uint32_t i = i0; i < i1; ++i) {
            while (s_end[lo] <= i) ++lo;
            list[base + i] = make_uint4(s_q[lo], i - s_beg[lo], s_end[lo] - s_beg[lo], s_ea[lo]);
        }
    }
    __syncthreads();
}

// --- Eq. (mode) ----------------------------------------------------------------------------------

// PC iff den * E^p * (3 n_png + k + E^p) <= num * (V_a E^p + 3 E_a E^p + 2 n_png E_a):
// Sec. 3.2's two traffic formulas (s_i = s_v = 4 B) multiplied through by E^p
// (so r^p E_a becomes the integer n_png E_a) and divided by 4.
__device__ __forceinline__ uint8_t analytic_mode(uint64_t k, uint64_t Ep, uint64_t npng, uint64_t Va, uint64_t Ea,
                                                 uint32_t num, uint32_t den) {
    if (Va == 0 || Ep == 0) return kModeNone;
    unsigned __int128 pc = (unsigned __int128)den * Ep * (unsigned __int128)(3 * npng + k + Ep);
    unsigned __int128 sc = (unsigned __int128)num *
                           ((unsigned __int128)Va * Ep + (unsigned __int128)3 * Ea * Ep + (unsigned __int128)2 * npng * Ea);
    return pc <= sc ? kModePC : kModeSC;
}

// The PC bytes of Sec. 3.2 are an integer: summed exactly (FP64 arithmetic is scarce on this GPU)
__device__ __forceinline__ unsigned long long pc_mode_bytes(uint64_t k, uint64_t Ep, uint64_t npng) {
    return 4ull * (3 * npng + k + Ep);
}
// The SC bytes 4 (V_a + 3 E_a + 2 r^p E_a), r^p = n_png / E^p, in integers: a whole number of bytes and
// two 32-bit digits of the fraction 8 rem / E^p (units of 2^-29 and 2^-61 bytes, rounded down), by long
// division (n_png E_a < 2^64 since E_a <= E^p < 2^32 and n_png <= E^p)
__device__ __forceinline__ unsigned long long sc_mode_bytes(uint32_t Ep, uint32_t npng, uint64_t Va, uint64_t Ea,
                                                            unsigned long long *d1, unsigned long long *d2) {
    const unsigned long long x = (unsigned long long)npng * Ea, qt = x / Ep, rm = x - qt * Ep;
    *d1 = (rm << 32) / Ep;
    *d2 = (((rm << 32) - *d1 * Ep) << 32) / Ep;
    return 4ull * (Va + 3 * Ea) + 8ull * qt;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Selector features of one partition in one iteration (shared by logging and inference):
// log1p V_a, log1p E_a, log1p E^p, r^p, log1p(bins in the row), log1p n_png, log1p k,
// and the log of Eq. (mode)'s cost ratio (PC cost / BW_PC over SC cost / BW_SC).
__device__ __forceinline__ void partition_features(uint64_t Va, uint64_t Ea, uint64_t Ep, uint64_t np, uint32_t k,
                                                   uint32_t row_bins, uint32_t num, uint32_t den, float f[8]) {
    double cpc = 4.0 * (double)(3 * np + k + Ep) * den;
    double csc = 4.0 * ((double)Va + 3.0 * (double)Ea + 2.0 * ((double)np / (double)Ep) * (double)Ea) * num;
    f[0] = log1pf((float)Va);
    f[1] = log1pf((float)Ea);
    f[2] = log1pf((float)Ep);
    f[3] = (float)((double)np / (double)Ep);
    f[4] = log1pf((float)row_bins);
    f[5] = log1pf((float)np);
    f[6] = log1pf((float)k);
    f[7] = (float)log(cpc / csc);
}

// Learned selector: MLP 8->32->32->1 (ReLU), lane j computes hidden unit j.
// Returns 2 (PC), 1 (SC) or 0xFF when the features are outside the training
// range (the caller then falls back to Eq. (mode)).  All lanes must call it.
// MLP selector forward pass for one partition by one warp (lane j = hidden unit j).  w is the parameter
// vector in the gpop_selector_set layout with W1 and W2 transposed, so that lanes read consecutive words.  Returns kModePC iff the predicted log(t_PC / t_SC) <= 0, or 0xFF when a feature lies outside
// the range seen in training (the caller then falls back to Eq. (mode)).
__device__ uint8_t learned_mode(const float *w, const float f[8], int lane) {
    const float *W1t = w, *b1 = W1t + 256, *W2t = b1 + 32, *b2 = W2t + 1024, *W3 = b2 + 32, *b3 = W3 + 32;
    const float *mean = b3 + 1, *sd = mean + 8, *fmin = sd + 8, *fmax = fmin + 8;
    bool in_range = true;
    float z[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        in_range &= (f[i] >= fmin[i]) && (f[i] <= fmax[i]);
        z[i] = (f[i] - mean[i]) / sd[i];
    }
    float h1 = b1[lane];
#pragma unroll
    for (int i = 0; i < 8; ++i) h1 = fmaf(W1t[i * 32 + lane], z[i], h1);
    h1 = fmaxf(h1, 0.f);
    float h2 = b2[lane];
#pragma unroll 8
    for (int i = 0; i < 32; ++i) h2 = fmaf(W2t[i * 32 + lane], __shfl_sync(0xffffffffu, h1, i), h2);
    h2 = fmaxf(h2, 0.f);
    float y = W3[lane] * h2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    y += b3[0];
    if (!in_range) return 0xFF;
    return y <= 0.f ? kModePC : kModeSC;
}

// Learned choice for partition q by one warp, from the gather-task statistics stamped `stamp` (the
// network read from global memory, transposed layout: coalesced); writes sel_mode[q].
__device__ void select_partition(const Params &p, uint32_t q, uint32_t stamp, int lane) {
    unsigned long long Va = 0, Ea = 0;
    for (uint32_t t = p.col_task[q] + lane; t < p.col_task[q + 1]; t += 32)
        if (__ldcg(&p.t_stamp[t]) == stamp) { Va += __ldcg(&p.t_va[t]); Ea += __ldcg(&p.t_ea[t]); }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Va += __shfl_xor_sync(0xffffffffu, Va, o);
        Ea += __shfl_xor_sync(0xffffffffu, Ea, o);
    }
    const uint64_t Ep = p.Ep[q], np = p.npng_p[q];
    uint8_t m = kModeNone;
    if (Va != 0 && Ep != 0) {
        float f[8];
        partition_features(Va, Ea, Ep, np, p.k, p.row_bin[q + 1] - p.row_bin[q], p.bw_num, p.bw_den, f);
        m = learned_mode(p.selector, f, lane);
    }
    if (lane == 0) p.sel_mode[q] = m;
}

// Programmatic dependent launch: the kernels of an iteration are launched so that each one's CTAs are
// placed on the SMs as the CTAs of the one before it exit, instead of after the whole grid has retired.
// Every one of them first waits until its predecessor in the stream has completed and its writes are
// visible (griddepcontrol.wait; an immediate return for an ordinary launch).  None triggers its successor
// early: successors placed while the predecessor still runs made an iteration slower.
#define GPOP_GRID_DEP() asm volatile("griddepcontrol.wait;\n" ::: "memory")

// Learned SC/PC choice for every partition (spec selector, Sec. 3.2's decision made by the MLP),
// for the first iteration of a run: one warp per partition computes V_a and E_a from the initial
// gather-task statistics (as k_plan does), the features and the forward pass, with the network staged
// in shared memory.  Writes kModePC / kModeSC, 0xFF for a fallback to Eq. (mode), or kModeNone.  Later
// iterations get their choices from the tail of k_gather (the last task of each column to finish).
constexpr int kSelectWarps = 8;
__global__ void __launch_bounds__(32 * kSelectWarps) k_select(Params p) {
    GPOP_GRID_DEP();
    __shared__ float s_w[GPOP_SELECTOR_PARAMS];
    for (int i = threadIdx.x; i < GPOP_SELECTOR_PARAMS; i += blockDim.x) s_w[i] = p.selector[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t prev = p.epoch - 1;
    for (uint32_t q = blockIdx.x * kSelectWarps + wid; q < p.k; q += gridDim.x * kSelectWarps) {
        unsigned long long Va = 0, Ea = 0;
        for (uint32_t t = p.col_task[q] + lane; t < p.col_task[q + 1]; t += 32)
            if (p.t_stamp[t] == prev) { Va += p.t_va[t]; Ea += p.t_ea[t]; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Va += __shfl_xor_sync(0xffffffffu, Va, o);
            Ea += __shfl_xor_sync(0xffffffffu, Ea, o);
        }
        const uint64_t Ep = p.Ep[q], np = p.npng_p[q];
        uint8_t m = kModeNone;
        if (Va != 0 && Ep != 0) {
            float f[8];
            partition_features(Va, Ea, Ep, np, p.k, p.row_bin[q + 1] - p.row_bin[q], p.bw_num, p.bw_den, f);
            m = learned_mode(s_w, f, lane);
        }
        if (lane == 0) p.sel_mode[q] = m;
    }
}

// --- initial frontier --------------------------------------------------------------------------

template <int ALGO>
__global__ void k_init(Params p) {
    if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->error = 0;  // device check flags, sticky for the run
    uint32_t nw = (p.V + 31) / 32;
    for (uint32_t wi = blockIdx.x * blockDim.x + threadIdx.x; wi < nw; wi += gridDim.x * blockDim.x) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            uint32_t g = wi * 32 + b;
            if (g >= p.V) break;
            uint32_t deg = p.rowptr[g + 1] - p.rowptr[g];
            bool act;
            uint32_t v, sv;
            if (ALGO == ALG_PR) {
                float x = 1.0f / (float)p.V;
                v = f2u(x);
                act = true;
                sv = f2u(deg ? x / (float)deg : 0.f);
            } else if (ALGO == ALG_PPR) {
                act = (g == p.source);
                v = f2u(act ? 1.f : 0.f);
                sv = act ? f2u(deg ? 1.f / (float)deg : 0.f) : kNull;
            } else if (ALGO == ALG_NIBBLE) {  // Alg. 4: PR = indicator of the seed, frontier = {seed}
                act = (g == p.source);
                v = f2u(act ? 1.f : 0.f);
                sv = act ? f2u(deg ? 1.f / (2.f * (float)deg) : 0.f) : kNull;
            } else if (ALGO == ALG_BFS) {
                act = (g == p.source);
                v = act ? g : kInf;
                p.lvl[g] = act ? 0u : kInf;
                sv = act ? g : kNull;
            } else if (ALGO == ALG_SSSP) {
                act = (g == p.source);
                v = act ? 0u : kInf;
                sv = act ? 0u : kNull;
            } else if (ALGO == ALG_MSBFS) {  // no source has reached anyone yet (k_msbfs_sources plants them)
                act = false;
                v = 0u;
                sv = kNull;
            } else {  // CC: own ID as label, everyone active
                act = true;
                v = g;
                sv = g;
            }
            p.val[g] = v;
            p.sval[g] = sv;
            if (act) word |= 1u << b;
        }
        p.bits[wi] = word;
    }
}

// Multi-source BFS: source j of the pass reaches its own vertex at level 0 (one thread: at most 32
// sources, and several may share a vertex).  Runs after k_init, before k_task_stats.
__global__ void k_msbfs_sources(Params p) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (uint32_t j = 0; j < p.nsrc; ++j) {
        const uint32_t g = p.msrc[j];
        p.val[g] |= 1u << j;
        p.lvl_ms[(uint64_t)j * p.V + g] = 0u;
        p.bits[g >> 5] |= 1u << (g & 31);
    }
    for (uint32_t j = 0; j < p.nsrc; ++j) p.sval[p.msrc[j]] = ~p.val[p.msrc[j]];  // message: complemented set
}

// frontier statistics of every gather task from the bitmap (used once, for the initial frontier)
__global__ void k_task_stats(Params p) {
    __shared__ uint32_t s_va[kGatherWarps];
    __shared__ unsigned long long s_ea[kGatherWarps];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < p.ngt; t += gridDim.x) {
        GatherTask gt = p.gtask[t];
        uint32_t va = 0;
        unsigned long long ea = 0;
        for (uint32_t d = gt.d0 + threadIdx.x; d < gt.d1; d += blockDim.x) {
            uint32_t g = (gt.q << p.shift) + d;
            if (g < p.V && ((p.bits[g >> 5] >> (g & 31)) & 1u)) {
                va++;
                ea += p.rowptr[g + 1] - p.rowptr[g];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            va += __shfl_xor_sync(0xffffffffu, va, o);
            ea += __shfl_xor_sync(0xffffffffu, ea, o);
        }
        if (lane == 0) { s_va[wid] = va; s_ea[wid] = ea; }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t a = 0;
            unsigned long long b = 0;
            for (int i = 0; i < kGatherWarps; ++i) { a += s_va[i]; b += s_ea[i]; }
            p.t_va[t] = a;
            p.t_ea[t] = b;
            p.t_res[t] = t == 0 ? __double2ull_rn(p.t_res0 * kResOne) : 0ull;  // a resumed run's first plan sees the saved L1 change
            p.t_stamp[t] = p.epoch;
        }
        __syncthreads();
    }
}

// --- plan: modes, actions, SC list, termination ------------------------------------------------

__global__ void __launch_bounds__(kPlanThreads) k_plan(Params p) {
    GPOP_GRID_DEP();
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_ub[kPlanThreads], s_ue[kPlanThreads], s_uq[kPlanThreads], s_uea[kPlanThreads];
    __shared__ unsigned long long s_v[kPlanThreads / 32], s_e[kPlanThreads / 32], s_sv[kPlanThreads / 32],
        s_se[kPlanThreads / 32], s_bp[kPlanThreads / 32];
    __shared__ unsigned long long s_r[kPlanThreads / 32];
    __shared__ unsigned long long s_f1[kPlanThreads / 32], s_f2[kPlanThreads / 32];
    __shared__ uint32_t s_ct[kPlanThreads + 1];  // the chunk's task offsets (col_task)
    __shared__ uint32_t s_pc[kPlanThreads / 32], s_sc[kPlanThreads / 32], s_nl[kPlanThreads / 32], s_fb[kPlanThreads / 32];
    __shared__ uint32_t s_cva[kPlanThreads];
    __shared__ unsigned long long s_cea[kPlanThreads];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t prev = p.epoch - 1;
    unsigned long long tv = 0, te = 0, tsv = 0, tse = 0, tbp = 0, tr = 0;  // tr: L1 change (fixed point)
    unsigned long long tf1 = 0, tf2 = 0;  // fractions of the SC model bytes (whole bytes: in tbp)
    uint32_t npc = 0, nsc = 0, nnull = 0, nfb = 0, sc_base = 0, pc_base = 0;

    uint32_t all_base = 0;
    // partitions in chunks of blockDim so the SC list can be compacted in order
    for (uint32_t base = 0; base < p.k; base += blockDim.x) {
        uint32_t q = base + threadIdx.x;
        uint8_t m = kModeNone;
        bool valid = q < p.k;
        uint64_t Va = 0, Ea = 0;
        uint32_t Ep = 0, np = 0;  // loaded before the task statistics, widened where used
        float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint8_t pcs = 0;
        if (valid) {
            Ep = p.Ep[q];
            np = p.npng_p[q];
            pcs = p.pc_state[q];
        }
        // V_a and E_a of the chunk's columns from the last iteration's gather-task statistics: the block
        // takes the chunk's tasks (contiguous, dozens for a hub column) together, each thread a run of
        // consecutive tasks with kPlanLoads loads in flight, and adds each column's share of its run into
        // per-column shared counters (integers: exact in any order)
        const uint32_t nq = min(blockDim.x, p.k - base);  // columns of the chunk
        s_cva[threadIdx.x] = 0u;
        s_cea[threadIdx.x] = 0ull;
        if (threadIdx.x < nq) s_ct[threadIdx.x] = p.col_task[base + threadIdx.x];
        if (threadIdx.x == 0) s_ct[nq] = p.col_task[base + nq];
        __syncthreads();
        {
            const uint32_t tlo = s_ct[0], thi = s_ct[nq];
            const uint32_t per = (thi - tlo + blockDim.x - 1) / blockDim.x;
            const uint32_t r0 = tlo + threadIdx.x * per, r1 = min(thi, r0 + per);
            // the column (within the chunk) of task r0: the last c with s_ct[c] <= r0
            uint32_t c = 0;
            if (r0 < r1) {
                uint32_t lo = 0, hi = nq - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (s_ct[mid] <= r0) lo = mid; else hi = mid - 1;
                }
                c = lo;
            }
            uint32_t cva = 0;
            unsigned long long cea = 0;
            for (uint32_t t = r0; t < r1; t += kPlanLoads) {
                uint32_t st[kPlanLoads], va[kPlanLoads];
                unsigned long long ea[kPlanLoads], rs[kPlanLoads];
#pragma unroll
                for (uint32_t u = 0; u < kPlanLoads; ++u) {
                    const bool in = t + u < r1;
                    st[u] = in ? __ldg(&p.t_stamp[t + u]) : ~prev;
                    va[u] = in ? __ldg(&p.t_va[t + u]) : 0u;
                    ea[u] = in ? __ldg(&p.t_ea[t + u]) : 0ull;
                    rs[u] = in ? __ldg(&p.t_res[t + u]) : 0ull;
                }
#pragma unroll
                for (uint32_t u = 0; u < kPlanLoads; ++u) {
                    if (t + u >= r1) break;
                    while (s_ct[c + 1] <= t + u) {  // task t + u starts a later column: flush this one
                        if (cva | cea) {
                            atomicAdd(&s_cva[c], cva);
                            atomicAdd(&s_cea[c], cea);
                        }
                        cva = 0;
                        cea = 0;
                        ++c;
                    }
                    if (st[u] == prev) {
                        cva += va[u];
                        cea += ea[u];
                        tr += rs[u];
                    }
                }
            }
            if (cva | cea) {
                atomicAdd(&s_cva[c], cva);
                atomicAdd(&s_cea[c], cea);
            }
        }
        __syncthreads();
        Va = s_cva[threadIdx.x];
        Ea = s_cea[threadIdx.x];
        if (valid) {
            tv += Va; te += Ea;
            if (Va == 0 || Ep == 0) m = kModeNone;
            else if (p.policy == GPOP_MODE_FORCE_SC) m = kModeSC;
            else if (p.policy == GPOP_MODE_FORCE_PC) m = kModePC;
            else m = analytic_mode(p.k, Ep, np, Va, Ea, p.bw_num, p.bw_den);
            if (m != kModeNone && p.log_both)
                partition_features(Va, Ea, Ep, np, p.k, p.row_bin[q + 1] - p.row_bin[q], p.bw_num, p.bw_den, f);
            if (p.log_both) {
                for (int i = 0; i < 8; ++i) p.feat[(uint64_t)q * 8 + i] = f[i];
                p.part_va[q] = (uint32_t)Va;
                p.part_ea[q] = Ea;
            }
        }
        if (p.policy == GPOP_MODE_LEARNED && p.selector && valid && m != kModeNone) {
            const uint8_t lm = p.sel_mode[q];  // k_select's choice; 0xFF: features outside the training range
            if (lm == 0xFF) nfb++;
            else if (lm != kModeNone) m = lm;
        }
        // interleaved scatter-gather: only this iteration's wave scatters; the others keep their frontier
        if (p.isg_w >= 2 && valid && q % p.isg_w != (p.iter - 1) % p.isg_w) m = kModeNone;
        if (valid) {
            p.mode[q] = m;
            if (m == kModePC) tbp += pc_mode_bytes(p.k, Ep, np);
            else if (m == kModeSC) {
                unsigned long long d1, d2;
                tbp += sc_mode_bytes(Ep, np, Va, Ea, &d1, &d2);
                tf1 += d1;
                tf2 += d2;
            }
            if (Va > 0) p.gflag[q] = p.epoch;  // active partitions are gathered (reInit of Alg. 2)
            npc += (m == kModePC);
            nsc += (m == kModeSC);
            if (m == kModeSC) {
                tsv += Va;
                tse += Ea;
            }
            uint8_t act = m == kModePC ? kActPC : (pcs ? kActNull : kActSkip);
            nnull += (act == kActNull);
            p.action[q] = act;
        }
        {  // PC partitions before q: the PC gather skips blocks whose source partitions are none of them
            uint32_t totp;
            uint32_t offp = block_excl_scan((valid && m == kModePC) ? 1u : 0u, s_warp, &totp);
            if (valid) p.pc_prefix[q] = pc_base + offp;
            pc_base += totp;
        }
        // SC scatter units: a partition's active edges are cut into ranges of about kScUnitEdges, each
        // scattered by one CTA (k_sc_segments has counted every segment's active edges, so a unit only
        // visits the segments its range overlaps)
        const uint32_t nu = (uint32_t)max(1ull, min((unsigned long long)((Ea + kScUnitEdges - 1) / kScUnitEdges), 65535ull));
        uint32_t total;
        const uint32_t nsc_u = (valid && m == kModeSC) ? nu : 0u;
        uint32_t off = block_excl_scan(nsc_u, s_warp, &total);
        if (total) write_units(p.sc_list, sc_base, q, nsc_u, off, total, (uint32_t)Ea, s_ub, s_ue, s_uq, s_uea);
        sc_base += total;
        if (p.log_both) {
            const uint32_t nall_u = (valid && m != kModeNone) ? nu : 0u;
            uint32_t off2 = block_excl_scan(nall_u, s_warp, &total);
            if (total) write_units(p.all_list, all_base, q, nall_u, off2, total, (uint32_t)Ea, s_ub, s_ue, s_uq, s_uea);
            all_base += total;
        }
    }
    // deterministic block reductions (fixed orders; integers exact)
    tv = warp_sum_u64(tv);
    te = warp_sum_u64(te);
    tsv = warp_sum_u64(tsv);
    tse = warp_sum_u64(tse);
    tbp = warp_sum_u64(tbp);
    tr = warp_sum_u64(tr);
    tf1 = warp_sum_u64(tf1);
    tf2 = warp_sum_u64(tf2);
    npc = __reduce_add_sync(0xffffffffu, npc);
    nsc = __reduce_add_sync(0xffffffffu, nsc);
    nnull = __reduce_add_sync(0xffffffffu, nnull);
    nfb = __reduce_add_sync(0xffffffffu, nfb);
    if (lane == 0) {
        s_v[wid] = tv; s_e[wid] = te; s_r[wid] = tr; s_f1[wid] = tf1; s_f2[wid] = tf2; s_sv[wid] = tsv; s_se[wid] = tse; s_bp[wid] = tbp;
        s_pc[wid] = npc; s_sc[wid] = nsc; s_nl[wid] = nnull; s_fb[wid] = nfb;
    }
    __syncthreads();
    __shared__ uint32_t s_done;
    if (threadIdx.x == 0) {
        constexpr int kNw = kPlanThreads / 32;  // k_plan runs one block of kPlanThreads
        unsigned long long a = 0, b = 0, sa = 0, sb = 0, bp = 0, rf = 0, f1 = 0, f2 = 0;
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll 4
        for (int i = 0; i < kNw; ++i) {
            a += s_v[i]; b += s_e[i]; sa += s_sv[i]; sb += s_se[i]; bp += s_bp[i]; rf += s_r[i];
            f1 += s_f1[i]; f2 += s_f2[i];
            c0 += s_pc[i]; c1 += s_sc[i]; c2 += s_nl[i]; c3 += s_fb[i];
        }
        const double r = (double)rf * kResUnit;
        uint32_t done = (a == 0) || (p.iter > p.max_iters);
        if ((p.algo == ALG_PR || p.algo == ALG_PPR) && p.iter > 1 && r < p.tol) done = 1;
        Control c;
        c.frontier_v = a; c.frontier_e = b; c.residual = r; c.model_bytes = (double)bp + (double)f1 * 0x1p-29 + (double)f2 * 0x1p-61;
        c.n_pc = c0; c.n_sc = c1; c.n_null = c2; c.done = done; c.n_fallback = c3; c.error = p.ctrl->error;
        c.n_sc_units = sc_base;
        p.pc_prefix[p.k] = pc_base;
        c.pad = 0;
        c.sc_v = sa;
        c.sc_e = sb;
        *p.ctrl = c;
        // read by the host after it has synchronised with the stream (the kernel's completion makes
        // the write visible)
        p.ctrl_snap[(p.iter - 1) & 1] = c;
        for (int i = 0; i < 8; ++i) p.counters[i] = 0;
        p.counters[7] = all_base;  // LOG_BOTH: size of all_list
        s_done = done;
    }
    __syncthreads();
    if (!s_done) {  // commit the PC-state of each data row only if this iteration runs
        for (uint32_t q = threadIdx.x; q < p.k; q += blockDim.x) p.pc_state[q] = p.mode[q] == kModePC;
        for (uint32_t t = threadIdx.x; t < p.ngt; t += blockDim.x) p.task_sc_cnt[t] = 0;
    }
}

// --- PC scatter (Alg. 3) -----------------------------------------------------------------------

// --- mbarriers and bulk copies (k_scatter_pc value staging, k_gather_pc buffers) ---------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) { return (uint32_t)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// makes the barrier initialisations visible to the asynchronous (bulk copy) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// 1-D bulk copy global -> shared (TMA engine): 16-byte aligned addresses, size a multiple of 16; the bytes
// are counted against the barrier's transaction count when they land
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// L2 policy that marks the lines it touches as first to evict: for data read exactly once, so that it does
// not push out lines prefetched for later use
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    return pol;
}
// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// One try with a suspend-time hint: the thread sleeps until the phase completes or about ns nanoseconds
// pass, instead of returning after the hardware's own short limit (so a waiting warp issues almost nothing)
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Waits for the completion of the barrier phase with the given parity: at most `limit` tries (each one
// sleeping up to sleep_ns, or the hardware's own limit when sleep_ns is 0) and at most kPcWaitNs in all;
// gives up early when another warp has raised *abort, and raises it (with the run's error flag) when its
// own tries or time run out.  Returns false when the caller must stop.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort, uint32_t *err,
                                          uint32_t limit = kPcSpinLimit, uint32_t sleep_ns = 0) {
    unsigned long long t0 = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        if (sleep_ns ? mbar_try_wait_sleep(bar, parity, sleep_ns) : mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        const unsigned long long now = globaltimer();
        if (it == 0) t0 = now;
        else if (now - t0 > kPcWaitNs) break;
    }
    *abort = 1;
    atomicOr(err, 1u);
    return false;
}

// Diagnostic of the bounded waits: one thread waits, through mbar_wait with `tries` polls, on a freshly
// initialised mbarrier whose first phase nothing completes (no arrival, no copy); the wait must give up
// and raise bit 0 of *err.  Bit 1 would mean the phase completed, which cannot happen.
__global__ void k_wait_probe(uint32_t tries, uint32_t *err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t abort;
    if (threadIdx.x != 0) return;
    abort = 0;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (mbar_wait(&bar, 0, &abort, err, tries)) atomicOr(err, 2u);
}

// Bounded wait used while leaving after an abort: lets copies still in flight land before the CTA exits.
// Should it run out too (a copy that never completes, which no test can cause without a fault), the CTA
// leaves with that copy still in flight; the run has reported GPOP_ERR_TIMEOUT by then.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kPcSpinLimit && !mbar_try_wait(bar, parity); ++it) {
    }
}

// --- PC scatter (Alg. 3) -----------------------------------------------------------------------

// One CTA per scatter task: a chunk of one partition's PNG row (Alg. 3 for a PC partition, or a row
// chunk refilled with NULL when the partition's data row must be cleared).  A PC task stages the
// partition's P message values in shared memory with one bulk copy (TMA; bounded mbarrier wait) and
// streams its chunk of the row: each thread reads eight 16-byte groups of 8 PNG source IDs ahead and
// writes the 8 values of each group as two 16-byte stores.
template <bool B16>
__global__ void __launch_bounds__(kScatterPcThreads) k_scatter_pc(Params p) {
    GPOP_GRID_DEP();
    extern __shared__ __align__(16) uint32_t s_val[];  // the partition's P message values (PC rows)
    __shared__ __align__(8) uint64_t s_bar;            // completion of the value copy
    __shared__ uint32_t s_task, s_ok;
    __shared__ unsigned long long s_t0;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    uint32_t phase = 0;  // parity of s_bar's current phase
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(&p.counters[p.counter_slot], 1u);
        __syncthreads();
        uint32_t t = s_task;
        __syncthreads();
        if (t >= p.nst) break;
        ScatterTask st = p.stask[t];
        // a shadow launch (LOG_BOTH) scatters every partition picked for this iteration into a
        // private buffer, to time PC mode where Eq. (mode) chose SC
        uint8_t act = p.dry ? (p.mode[st.p] != kModeNone ? kActPC : kActSkip) : p.action[st.p];
        if (act == kActSkip) continue;
        if (p.t_task && threadIdx.x == 0) s_t0 = globaltimer();
        if (act == kActPC && st.first && !p.dry) {
            // the partition's messages reach every column of its bin row
            for (uint32_t b = p.row_bin[st.p] + threadIdx.x; b < p.row_bin[st.p + 1]; b += blockDim.x) {
                uint32_t q = p.bin_q[b];
                p.gflag[q] = p.epoch;
                p.gflag_pc[q] = p.epoch;
            }
        }
        const uint32_t vbase = st.p << p.shift;
        if (act == kActPC) {
            // stage the partition's values (NULL for inactive sources): the 16-byte multiple by one bulk
            // copy, the last (V mod 4) values of a ragged final partition by plain loads.  The barrier at the
            // top of the loop ordered every read of the previous task's values before this copy.
            const uint32_t wv = min(p.P, p.V - vbase), wa = wv & ~3u;
            if (threadIdx.x == 0) {
                s_ok = 1;
                if (wa) {
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    mbar_arrive_expect_tx(&s_bar, wa * 4u);
                    bulk_g2s(s_val, p.sval + vbase, wa * 4u, &s_bar);
                }
            }
            for (uint32_t c = wa + threadIdx.x; c < wv; c += blockDim.x) s_val[c] = p.sval[vbase + c];
            if (wa && threadIdx.x == 0) {
                uint32_t it = 0;
                while (it < kPcSpinLimit && !mbar_try_wait(&s_bar, phase)) ++it;
                if (it == kPcSpinLimit) {
                    atomicOr(&p.ctrl->error, 1u);
                    mbar_drain(&s_bar, phase);
                    s_ok = 0;
                }
            }
            if (wa) phase ^= 1u;
            __syncthreads();
            if (!s_ok) return;  // the run reports the error; the copy has landed or been waited out
        }
        const uint32_t stride = blockDim.x * 8;
        for (uint32_t i0 = st.beg + threadIdx.x * 8; i0 < st.end; i0 += 8 * stride) {
            uint4 sx[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {  // up to eight independent 16-byte loads in flight
                const uint32_t i = i0 + u * stride;
                sx[u] = (act == kActPC && i < st.end) ? *reinterpret_cast<const uint4 *>(p.png + i)
                                                       : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t i = i0 + u * stride;
                if (i >= st.end) break;
                uint4 o0, o1;
                if (act == kActPC) {  // padding slots hold source 0: staged, never gathered
                    const uint4 sv = sx[u];
                    o0.x = s_val[sv.x & 0xFFFFu];
                    o0.y = s_val[sv.x >> 16];
                    o0.z = s_val[sv.y & 0xFFFFu];
                    o0.w = s_val[sv.y >> 16];
                    o1.x = s_val[sv.z & 0xFFFFu];
                    o1.y = s_val[sv.z >> 16];
                    o1.z = s_val[sv.w & 0xFFFFu];
                    o1.w = s_val[sv.w >> 16];
                } else {
                    o0 = make_uint4(kNull, kNull, kNull, kNull);
                    o1 = o0;
                }
                if (B16) {  // 8 BF16 slots in one 16-byte store (slot 2k in the low half of word k)
                    const uint4 h = make_uint4(to_bf16(o0.x) | (to_bf16(o0.y) << 16), to_bf16(o0.z) | (to_bf16(o0.w) << 16),
                                               to_bf16(o1.x) | (to_bf16(o1.y) << 16), to_bf16(o1.z) | (to_bf16(o1.w) << 16));
                    *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(p.pdata) + i) = h;
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(p.pdata + i);
                    dst[0] = o0;
                    dst[1] = o1;
                }
            }
        }
        if (p.t_task) {
            __syncthreads();
            if (threadIdx.x == 0) p.t_task[t] = globaltimer() - s_t0;
        }
    }
}

// --- SC scatter (Alg. 2 scatter in source-centric mode) ---------------------------------------

// Active out-edges of every 1024-vertex segment of the partitions scattered in SC mode this iteration (of
// every scattered partition when a LOG_BOTH shadow pass times both modes), one warp per segment from the
// frontier bits and the row offsets; the SC scatter's units find their edge ranges in these counts.
__global__ void k_sc_segments(Params p) {
    GPOP_GRID_DEP();
    const uint32_t nseg = (p.P + 1023) / 1024;
    const int lane = threadIdx.x & 31;
    const uint64_t nw = (uint64_t)p.k * nseg, step = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t wg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg < nw; wg += step) {
        const uint32_t q = (uint32_t)(wg / nseg), si = (uint32_t)(wg % nseg);
        const uint8_t m = p.mode[q];
        if (p.log_both ? m == kModeNone : m != kModeSC) continue;
        const uint32_t gend = min((q << p.shift) + p.P, p.V);
        const uint32_t gw = (q << p.shift) + si * 1024 + (uint32_t)lane * 32;
        uint32_t word = gw < gend ? p.bits[gw >> 5] : 0u;
        if (gw < gend && gend - gw < 32) word &= (1u << (gend - gw)) - 1u;
        uint32_t cnt = 0;
        if (word == 0xFFFFFFFFu) {
            cnt = p.rowptr[gw + 32] - p.rowptr[gw];
        } else {
            while (word) {
                const uint32_t u = gw + (uint32_t)(__ffs(word) - 1);
                word &= word - 1;
                cnt += p.rowptr[u + 1] - p.rowptr[u];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) p.sc_seg[(uint64_t)q * kScSegs + si] = cnt;
    }
}

// One CTA per work unit: about kScUnitEdges consecutive active edges of one SC partition (in the order of
// its active vertices), or all of a partition with fewer.  The unit passes over the segments before its
// range (their active-edge counts come from k_sc_segments); for each segment it overlaps, all threads
// build the segment's active vertices in ascending order with the prefix of their out-degrees (four
// vertices per thread), then expand the unit's edges one per thread; each pair goes to the sub-bin of its
// (partition, gather task) at a cursor bumped once per distinct sub-bin per warp.  A partition of one unit
// keeps its cursors in shared memory and publishes the counts at the end; the units of a split partition
// bump global cursors (zero at rest), and the last unit to finish publishes the counts and resets them.
template <int ALGO, bool B16>
__global__ void __launch_bounds__(kScatterThreads) k_scatter_sc(Params p) {
    GPOP_GRID_DEP();
    extern __shared__ uint32_t s_cursor[];  // per sub-bin of the row: its next free slot (a partition of one unit)
                                            // or its first slot (a split partition, cursors in global memory)
    // the current segment's active vertices, ascending: exclusive prefix of their out-degrees, first
    // out-edge (row offset) and message value (scatterFunc)
    __shared__ uint32_t s_pref[1025], s_row[1024], s_msg[1024];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_task, s_last;
    __shared__ unsigned long long s_t0;
    const int lane = threadIdx.x & 31;
    const uint32_t nunits = *p.list_count;
    const uint32_t nseg = (p.P + 1023) / 1024;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(&p.counters[p.counter_slot], 1u);
        __syncthreads();
        uint32_t t = s_task;
        __syncthreads();
        if (t >= nunits) break;
        const uint4 un = p.list[t];  // partition, unit, units, active edges
        const uint32_t part = un.x;
        const bool split = un.z > 1;
        // active-edge range of this unit (in the order of the partition's active vertices)
        const uint64_t ua = split ? (uint64_t)un.w * un.y / un.z : 0ull;
        const uint64_t ub = split ? (uint64_t)un.w * (un.y + 1) / un.z : ~0ull;
        if (p.t_task && threadIdx.x == 0) s_t0 = globaltimer();
        const uint32_t rb0 = p.row_sub[part], nbr = p.row_sub[part + 1] - rb0;
        // the row's sub-bin first slots are staged when the unit has at least as many edges as the row has
        // sub-bins (and always for a split partition); otherwise cursors count from 0 and the leader of each
        // warp's group looks its sub-bin up
        const bool staged = split || un.w >= nbr;
        for (uint32_t i = threadIdx.x; i < nbr; i += blockDim.x) s_cursor[i] = staged ? p.sub_cap[rb0 + i] : 0u;
        uint32_t *gcur = p.sc_gcur + rb0;  // a split partition's cursors (relative to the sub-bin's first slot)
        const uint32_t g0 = part << p.shift;
        const uint32_t gend = min(g0 + p.P, p.V);
        uint64_t run0 = 0;  // active edges of the partition before this segment
        for (uint32_t si = 0; si < nseg && run0 < ub; ++si) {
            const uint32_t seg_e = p.sc_seg[(uint64_t)part * kScSegs + si];  // the same for every thread
            if (seg_e == 0 || run0 + seg_e <= ua) {  // nothing to scatter here
                run0 += seg_e;
                continue;
            }
            // this segment's active vertices (thread i: vertices 4i .. 4i+3 of the segment) and the
            // exclusive prefix of their out-degrees
            const uint32_t v0 = g0 + si * 1024 + threadIdx.x * 4;
            uint32_t nib = 0;
            if (v0 < gend) {
                nib = (p.bits[v0 >> 5] >> (v0 & 31)) & 0xFu;
                if (gend - v0 < 4) nib &= (1u << (gend - v0)) - 1u;
            }
            uint32_t rp[5] = {0, 0, 0, 0, 0}, cnt = 0, esum = 0;
            if (nib) {
                rp[4] = p.rowptr[min(v0 + 4, p.V)];
                if (v0 + 4 <= p.V) {
                    const uint4 r = *reinterpret_cast<const uint4 *>(p.rowptr + v0);
                    rp[0] = r.x; rp[1] = r.y; rp[2] = r.z; rp[3] = r.w;
                } else {
                    for (uint32_t c = 0; c < 4; ++c) rp[c] = v0 + c <= p.V ? p.rowptr[v0 + c] : rp[4];
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if ((nib >> c) & 1u) {
                        ++cnt;
                        esum += rp[c + 1] - rp[c];
                    }
            }
            uint32_t nact, total;
            uint32_t k = block_excl_scan(cnt, s_warp, &nact);
            uint32_t ek = block_excl_scan(esum, s_warp, &total);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((nib >> c) & 1u) {  // list entry k: edge prefix, row offset, message value
                    s_pref[k] = ek;
                    s_row[k] = rp[c];
                    s_msg[k] = p.sval[v0 + c];
                    ++k;
                    ek += rp[c + 1] - rp[c];
                }
            if (threadIdx.x == 0) s_pref[nact] = total;
            __syncthreads();
            // this segment's active edges [run0, run0 + total) that belong to the unit
            const uint64_t seg_lo = max(ua, run0), seg_hi = min(ub, run0 + total);
            const uint32_t e_lo = seg_lo < seg_hi ? (uint32_t)(seg_lo - run0) : 0u;
            const uint32_t e_hi = seg_lo < seg_hi ? (uint32_t)(seg_hi - run0) : 0u;
            // expand the active edges, one thread per edge
            for (uint32_t base = e_lo; base < e_hi; base += blockDim.x) {
                uint32_t e = base + threadIdx.x;
                bool live = e < e_hi;
                uint32_t lb = 0xFFFFFFFFu, dloc = 0, val = 0, slot = 0;
                if (live) {
                    uint32_t lo = 0, hi = nact;  // largest i with s_pref[i] <= e
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (s_pref[mid] <= e) lo = mid; else hi = mid;
                    }
                    const uint32_t edge = s_row[lo] + (e - s_pref[lo]);
                    const uint32_t dst = p.col[edge];
                    lb = p.esub[edge];
                    dloc = dst & (p.P - 1);
                    val = s_msg[lo];
                    if (ALGO == ALG_SSSP) val = Op<ALGO>::weigh(val, p.w[edge]);
                }
                // warp-aggregated insertion: one cursor bump per distinct bin in the warp
                uint32_t peers = __match_any_sync(0xffffffffu, lb);
                int leader = __ffs(peers) - 1;
                uint32_t rank = __popc(peers & ((1u << lane) - 1));
                uint32_t basepos = 0;
                if (live && lane == leader)
                    basepos = split    ? s_cursor[lb] + atomicAdd(&gcur[lb], (uint32_t)__popc(peers))
                              : staged ? atomicAdd(&s_cursor[lb], (uint32_t)__popc(peers))
                                       : p.sub_cap[rb0 + lb] + atomicAdd(&s_cursor[lb], (uint32_t)__popc(peers));
                basepos = __shfl_sync(0xffffffffu, basepos, leader);
                if (live) {
                    slot = basepos + rank;
                    if (B16) reinterpret_cast<uint32_t *>(p.scpair)[slot] = dloc | (to_bf16(val) << 16);
                    else p.scpair[slot] = make_uint2(dloc, val);
                }
            }
            run0 += total;
            __syncthreads();
        }
        // publish counts and the 2-level active list (gPartList = gflag, binPartList = the gather
        // task's list of fresh SC bins); a split partition publishes once, from its last unit
        bool publish = !split;
        if (split) {
            if (threadIdx.x == 0) {
                __threadfence();
                s_last = atomicAdd(&p.sc_udone[part], 1u) == un.z - 1;
            }
            __syncthreads();
            publish = s_last != 0;
            if (publish) __threadfence();
        }
        if (publish) {
            for (uint32_t i = threadIdx.x; i < nbr; i += blockDim.x) {
                const uint32_t c = split    ? atomicExch(&gcur[i], 0u)
                                   : staged ? s_cursor[i] - p.sub_cap[rb0 + i]
                                            : s_cursor[i];
                if (c && !p.dry) {
                    uint32_t b = rb0 + i;
                    p.sccnt[b] = c;
                    uint32_t tsk = p.sub_task[b];
                    p.gflag[p.gtask[tsk].q] = p.epoch;
                    uint32_t pos = atomicAdd(&p.task_sc_cnt[tsk], 1u);
                    p.task_sc_list[p.task_sub_ptr[tsk] + pos] = b;
                }
            }
            if (split && threadIdx.x == 0) p.sc_udone[part] = 0;
        }
        __syncthreads();
        if (p.t_task && threadIdx.x == 0) {  // CTA time of the partition (units add up)
            const unsigned long long dt = globaltimer() - s_t0;
            if (split) atomicAdd(&p.t_task[part], dt);
            else p.t_task[part] = dt;
        }
    }
}

// --- gather + filter ---------------------------------------------------------------------------


// 32-bit shared-memory accesses at explicit shared addresses (the fold's addresses stay 32-bit; volatile
// keeps them in program order, which the read-modify-writes of consecutive rounds rely on).
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds16(uint32_t a) {
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) { asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v)); }

// Serial fold of one lane's K destination entries (its K consecutive positions of the round, held in
// registers as K / 4 quads), in batches of 8: the batch's message values are loaded first (independent
// shared loads), runs of equal destination are then found in registers, and the complete inner runs are
// folded into the accumulator with batched read-modify-writes (inner runs of a lane have distinct
// destinations, and no other lane or warp touches them).  A position that ends no inner run does its
// read-modify-write on a scratch word past the value buffer's padding slot (never copied into, never
// read for a result): fewer instructions than predicating the shared accesses.  Entries are sorted by destination, so a
// position belongs to the lane's first run exactly when its destination is the first one, fd; head follows
// that run's value.  Padding entries repeat their range's last destination and read the padding value slot
// (the identity), so they fold as no-ops.  NULL messages are skipped when NUL (SSSP, PPR, Nibble, and
// PageRank while some partition is not PC); SSSP adds each entry's edge weight (applyWeight of Alg. 7).
// stage and acc are shared-memory addresses.
template <int ALGO, bool B16, uint32_t K, bool NUL>
__device__ __forceinline__ void pc_lane(const uint4 (&E)[4], const int4 (&W)[4], uint32_t stage, uint32_t acc,
                                        uint32_t &fd, uint32_t &head, uint32_t &run_d, uint32_t &run_v) {
    using O = Op<ALGO>;
    static_assert(K == 4 || K == 8 || K == 16, "lanes fold 4, 8 or 16 entries per round");
    constexpr uint32_t HB = K < 8 ? K : 8;  // entries per batch
#pragma unroll
    for (uint32_t hb = 0; hb < K; hb += HB) {
        uint32_t ee[HB];
        int32_t ww[HB];
#pragma unroll
        for (uint32_t qq = 0; qq < HB / 4; ++qq) {
            const uint4 e4 = E[hb / 4 + qq];
            ee[4 * qq] = e4.x; ee[4 * qq + 1] = e4.y; ee[4 * qq + 2] = e4.z; ee[4 * qq + 3] = e4.w;
            const int4 w4 = W[hb / 4 + qq];
            ww[4 * qq] = w4.x; ww[4 * qq + 1] = w4.y; ww[4 * qq + 2] = w4.z; ww[4 * qq + 3] = w4.w;
        }
        uint32_t x[HB];
#pragma unroll
        for (uint32_t i = 0; i < HB; ++i) {
            if (B16) {  // BF16 values staged as 16-bit words
                const uint32_t h = lds16(stage + (ee[i] & 0xFFFFu) * 2u);
                x[i] = (NUL && h == kNull16) ? kNull : from_bf16(h);
            } else {
                x[i] = lds32(stage + (ee[i] & 0xFFFFu) * 4u);
            }
        }
        // ra: accumulator word of an inner run that ends at this position, else the scratch word
        const uint32_t kNoRun = stage + (kPcBlock + 1) * 4u;
        uint32_t ra[HB], fv[HB];
#pragma unroll
        for (uint32_t i = 0; i < HB; ++i) {
            // NULL (0xFFFFFFFF) is the identity of min and of AND, so BFS, CC and multi-source BFS fold it as is
            const uint32_t v = (!NUL || x[i] != kNull) ? O::weigh(x[i], ww[i]) : O::identity();
            const uint32_t d = ee[i] >> 16;
            if (hb == 0 && i == 0) {
                fd = run_d = d;
                run_v = v;
                ra[0] = kNoRun;
                fv[0] = O::identity();
                continue;
            }
            const bool ch = d != run_d, first = run_d == fd;
            ra[i] = (ch && !first) ? acc + run_d * 4u : kNoRun;
            fv[i] = run_v;
            head = first ? run_v : head;
            const uint32_t joined = O::combine(run_v, v);
            run_v = ch ? v : joined;
            run_d = d;
        }
        // read-modify-writes of the inner runs that end in this batch
        uint32_t old[HB];
#pragma unroll
        for (uint32_t i = 0; i < HB; ++i) old[i] = lds32(ra[i]);
#pragma unroll
        for (uint32_t i = 0; i < HB; ++i) sts32(ra[i], O::combine(old[i], fv[i]));
    }
}

// One warp round: n <= kPcRound positions (a multiple of 16), sorted by destination, all inside this
// warp's destination slice of the block, folded by the n / K lanes that hold them.  A lane's last run is
// continued by the next lane's first run when they share the destination: the next lane adds it to its
// first run and writes the sum, unless its whole range is that run, in which case one segmented warp scan
// (keyed by destination) carries the sum on.  Every complete run is folded into the accumulator directly:
// a run cut by the round's end continues in the warp's next round, folded after this part.
template <int ALGO, bool B16, uint32_t K, bool NUL>
__device__ __forceinline__ void pc_round(const uint4 (&E)[4], const int4 (&W)[4], uint32_t n, uint32_t stage,
                                         uint32_t acc, int lane) {
    using O = Op<ALGO>;
    uint32_t fd = kSent, head = O::identity(), run_d = kSent, run_v = O::identity();
    if ((uint32_t)lane * K < n) pc_lane<ALGO, B16, K, NUL>(E, W, stage, acc, fd, head, run_d, run_v);
    const uint32_t ld = run_d;
    const bool uni = ld == fd;  // all K positions share one destination (or the lane is idle: kSent)
    uint32_t S = run_v;
    if (__any_sync(0xffffffffu, uni && ld != kSent)) {  // a run spans a whole lane: scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t vu = __shfl_up_sync(0xffffffffu, S, o);
            const uint32_t du = __shfl_up_sync(0xffffffffu, ld, o);
            if (lane >= o && du == ld) S = O::combine(vu, S);
        }
    }
    const uint32_t prev_S = __shfl_up_sync(0xffffffffu, S, 1);
    const uint32_t prev_d = __shfl_up_sync(0xffffffffu, ld, 1);
    const uint32_t next_fd = __shfl_down_sync(0xffffffffu, fd, 1);
    if (!uni && fd != kSent) {  // first run ends inside this lane
        const uint32_t hv = (lane > 0 && prev_d == fd) ? O::combine(prev_S, head) : head;
        const uint32_t a = acc + fd * 4u;
        sts32(a, O::combine(lds32(a), hv));
    }
    if (ld != kSent && (lane == 31 || next_fd != ld)) {  // last run ends here
        const uint32_t a = acc + ld * 4u;
        sts32(a, O::combine(lds32(a), S));
    }
}

// Loads lane `lane`'s entries (and SSSP weights) of the round [s, s + n) of the lane-interleaved layout:
// quad j of the lane at s + (j * n / K + lane) * 4, K = pc_round_k(n); lanes past n / K and quads past
// K / 4 get zeros (never folded).  Streamed once: no L1 allocation.
__device__ __forceinline__ uint4 ldg_stream(const uint32_t *ptr) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(ptr));
    return r;
}
__device__ __forceinline__ void pc_load_round(const uint32_t *base, uint32_t s, uint32_t n, int lane, uint4 (&R)[4]) {
    const uint32_t K = pc_round_k(n), nl = n / K;
#pragma unroll
    for (uint32_t j = 0; j < 4; ++j)
        R[j] = (j < K / 4 && (uint32_t)lane < nl) ? ldg_stream(base + s + (j * nl + (uint32_t)lane) * 4)
                                                  : make_uint4(0, 0, 0, 0);
}
// Bulk prefetch of [ptr, ptr + bytes) into L2 (one instruction, no completion to wait for): 16-byte aligned
// address, size a multiple of 16
__device__ __forceinline__ void bulk_prefetch_l2(const void *ptr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(ptr), "r"(bytes) : "memory");
}

// Barrier 1 joins the consumer warps of k_gather_pc (the producer warp never takes part)
__device__ __forceinline__ void pc_consumers_sync() {
    asm volatile("bar.sync 1, %0;\n" ::"n"(kPcGatherWarps * 32) : "memory");
}
// the same barrier, returning whether any consumer thread passed a true predicate
__device__ __forceinline__ bool pc_consumers_or(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "n"(kPcGatherWarps * 32)
        : "memory");
    return r != 0;
}

// A PC gather task handed from the producer warp to the consumer warps of k_gather_pc
struct PcSlot {
    uint4 tk;                                   // column, first block, end block, partial slot (or kNull)
    uint32_t state;                             // 1: a task, 2: no task left
    uint32_t nb, na;                            // blocks of the task, blocks holding a PC message this iteration
    uint32_t run[kPcTaskBlocks + 1];            // bin runs of each block
    uint32_t nval[kPcTaskBlocks];               // staged values of each block
    uint32_t sp[kPcTaskBlocks * (kPcGatherWarps + 1)];  // each block's entry splits, one range per consumer warp
    uint32_t blist[kPcTaskBlocks];              // the active blocks, in order
};

// Copies n words from global to shared memory with one warp, 16 loads in flight per lane
__device__ __forceinline__ void warp_copy(uint32_t *dst, const uint32_t *src, uint32_t n, int lane) {
    constexpr uint32_t U = 16;
    for (uint32_t i0 = 0; i0 < n; i0 += 32 * U) {
        uint32_t v[U];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * 32 + (uint32_t)lane;
            v[u] = i < n ? src[i] : 0u;
        }
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * 32 + (uint32_t)lane;
            if (i < n) dst[i] = v[u];
        }
    }
}

// Producer warp of k_gather_pc: takes the tasks (largest first, from a device counter), describes each one
// in a task slot for the consumers, and stages the message values of the task's active blocks, one block
// per value buffer: once the consumers have released the buffer (its "empty" mbarrier), the block's bin
// runs are bulk-copied (TMA) into it, counted in on its "full" mbarrier.  The bins are read in order, as
// the paper's gather streams bin[:][q].  Waits are bounded; an abort stops the issue and every copy still
// in flight is waited out before the warp leaves.
template <bool B16>
__device__ void pc_producer(const Params &p, PcSlot *slots, uint64_t *full, uint64_t *empty, uint64_t *tfull,
                            uint64_t *tempty, uint32_t *stage, uint32_t nbuf, volatile uint32_t *abort, int lane) {
    constexpr uint32_t kB = B16 ? 2u : 4u, kSp = kPcGatherWarps + 1, kStageWords = kPcBlock + 4;
    const bool pc_skip = p.pc_skip != 0;
    uint32_t issued = 0;  // blocks staged so far: buffer issued % nbuf, use issued / nbuf
    bool ok = true;
    const uint64_t pol = l2_evict_first_policy();
    for (uint32_t n = 0; ok; ++n) {  // n: tasks handed over
        const uint32_t ts = n & 1;
        PcSlot &sl = slots[ts];
        if (n >= 2 && !__all_sync(0xffffffffu, mbar_wait(&tempty[ts], ((n >> 1) - 1) & 1u, abort, &p.ctrl->error, kPcSpinLimit, kPcSleepNs))) {
            ok = false;
            break;
        }
        uint32_t state = 2, t = 0;
        uint4 tk = make_uint4(0, 0, 0, 0);
        if (lane == 0) {
            for (;;) {  // the next task whose column received PC messages this iteration
                t = atomicAdd(&p.counters[5], 1u);
                if (t >= p.npct || *abort) break;
                tk = p.pc_task[t];
                if (p.gflag_pc[tk.x] == p.epoch) {
                    state = 1;
                    break;
                }
            }
        }
        state = __shfl_sync(0xffffffffu, state, 0);
        t = __shfl_sync(0xffffffffu, t, 0);
        tk.x = __shfl_sync(0xffffffffu, tk.x, 0);
        tk.y = __shfl_sync(0xffffffffu, tk.y, 0);
        tk.z = __shfl_sync(0xffffffffu, tk.z, 0);
        tk.w = __shfl_sync(0xffffffffu, tk.w, 0);
        uint32_t na = 0;
        if (state == 1) {
            const uint32_t nb = tk.z - tk.y;
            const uint64_t tsp = (uint64_t)p.pc_tsp[t] * kSp;
            warp_copy(sl.run, p.pc_blk_run + tk.y, nb + 1, lane);
            warp_copy(sl.nval, p.pc_blk_nval + tk.y, nb, lane);
            warp_copy(sl.sp, p.pc_wsp + tsp, nb * kSp, lane);
            // a block only holds NULLs unless one of its source partitions sent PC messages this iteration
            bool act = false;
            if ((uint32_t)lane < nb) {
                act = true;
                if (pc_skip) {
                    const uint2 pr = p.pc_blk_prange[tk.y + lane];
                    act = p.pc_prefix[pr.y + 1] != p.pc_prefix[pr.x];
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, act);
            if (act) sl.blist[__popc(m & ((1u << lane) - 1u))] = lane;
            na = __popc(m);
            if (lane == 0) {
                sl.tk = tk;
                sl.nb = nb;
                sl.na = na;
            }
        }
        if (lane == 0) sl.state = state;
        __threadfence_block();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tfull[ts]);
        if (state != 1) break;
        for (uint32_t j = 0; j < na; ++j, ++issued) {
            const uint32_t b = issued % nbuf, u = issued / nbuf;
            if (u > 0 && !__all_sync(0xffffffffu, mbar_wait(&empty[b], (u - 1) & 1u, abort, &p.ctrl->error, kPcSpinLimit, kPcSleepNs))) {
                ok = false;
                break;
            }
            const uint32_t i = sl.blist[j], r0 = sl.run[i], r1 = sl.run[i + 1];
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive_expect_tx(&full[b], sl.nval[i] * kB);
            }
            char *dst = reinterpret_cast<char *>(stage + b * kStageWords);
            // the block's bin runs (row-major source slot, length, offset in the block; multiples of 4 values,
            // so 16-byte aligned), eight descriptor loads in flight per lane; the values are read once, so
            // their L2 lines go first (the consumers' entries prefetched into L2 stay)
            for (uint32_t r = r0; r < r1; r += 32 * 8) {
                uint4 run[8];
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u) {
                    const uint32_t rr = r + u * 32 + (uint32_t)lane;
                    run[u] = rr < r1 ? p.pc_runs[rr] : make_uint4(0, 0, 0, 0);
                }
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u)
                    if (r + u * 32 + (uint32_t)lane < r1)
                        bulk_g2s_hint(dst + (size_t)run[u].z * kB,
                                      reinterpret_cast<const char *>(p.pdata) + (size_t)run[u].x * kB, run[u].y * kB,
                                      &full[b], pol);
            }
        }
    }
    // leave no copy in flight: the last phase armed on each buffer has completed (at once, normally)
    for (uint32_t b = 0; b < nbuf && b < issued; ++b) {
        const uint32_t last = (issued - 1 - b) / nbuf;  // last use of buffer b
        if (lane == 0) mbar_drain(&full[b], last & 1u);
    }
    __syncwarp();
}

// Consumer warp w of k_gather_pc: for every task, folds its entries of each active block (those of its
// destination range [D_w, D_w+1), the same in every block of the task, cut at build time so that no two
// warps ever touch one destination) into the shared column accumulator, round by round, with the next
// round's entries already loading into registers and its entries of the next block being fetched into
// L2; then all consumers write the column's result (or the task's partial vector) and reset the
// accumulator.
template <int ALGO, bool B16>
__device__ void pc_consumer(const Params &p, const PcSlot *slots, uint64_t *full, uint64_t *empty, uint64_t *tfull,
                            uint64_t *tempty, const uint32_t *stage, uint32_t *acc, uint32_t nbuf,
                            volatile uint32_t *abort, int lane, int w) {
    using O = Op<ALGO>;
    constexpr uint32_t kSp = kPcGatherWarps + 1, kStageWords = kPcBlock + 4;
    const bool chk = p.pc_skip != 0;  // some partition is not PC: NULL messages are possible
    const uint32_t acc_o = smem_addr(acc);
    uint32_t used = 0;                // blocks consumed: buffer used % nbuf, use used / nbuf
    for (uint32_t n = 0;; ++n) {
        const uint32_t ts = n & 1;
        const PcSlot &sl = slots[ts];
        bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[ts], (n >> 1) & 1u, abort, &p.ctrl->error, kPcSpinLimit, kPcSleepNs));
        const uint32_t state = ok ? sl.state : 2u;
        if (pc_consumers_or(state != 1)) break;  // all consumers leave together
        const uint32_t na = sl.na;
        // cursor over this warp's rounds in the task's active blocks: the next round to load into registers
        struct Cur {
            uint32_t j, s, e;  // active block, entries [s, e) of this warp's range left in it
        };
        auto seek = [&](Cur &c) {
            for (; c.j < na; ++c.j) {
                const uint32_t i = sl.blist[c.j];
                c.s = sl.sp[i * kSp + w];
                c.e = sl.sp[i * kSp + w + 1];
                if (c.s < c.e) break;
            }
        };
        // this warp's entries (and SSSP weights) of active block j, bulk-prefetched into L2 one block ahead
        // of their fold (the entries are 16-byte aligned and padded to whole 16-entry groups); further
        // ahead, the stream of other reads evicts part of them before use
        auto prefetch_block = [&](uint32_t j) {
            if (lane == 0 && j < na) {
                const uint32_t i = sl.blist[j], s = sl.sp[i * kSp + w], e = sl.sp[i * kSp + w + 1];
                if (s < e) {
                    bulk_prefetch_l2(p.pe + s, (e - s) * 4u);
                    if (ALGO == ALG_SSSP) bulk_prefetch_l2(p.pw + s, (e - s) * 4u);
                }
            }
        };
        prefetch_block(0);
        Cur c{0, 0, 0};
        seek(c);
        uint4 R[4];
        if (c.j < na) pc_load_round(p.pe, c.s, min(c.e - c.s, kPcRound), lane, R);
        for (uint32_t j = 0; j < na; ++j, ++used) {
            const uint32_t b = used % nbuf;
            prefetch_block(j + 1);
            // every consumer waits for every block, so that none is ever more than nbuf blocks ahead
            if (ok && !__all_sync(0xffffffffu, mbar_wait(&full[b], (used / nbuf) & 1u, abort, &p.ctrl->error, kPcSpinLimit, kPcSleepNs))) ok = false;
            const uint32_t vals = smem_addr(stage + b * kStageWords);
            while (ok && c.j == j) {
                uint4 E[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) E[q] = R[q];
                const uint32_t cs = c.s, cn = min(c.e - c.s, kPcRound);
                c.s += cn;
                if (c.s >= c.e) {
                    ++c.j;
                    seek(c);
                }
                if (c.j < na) pc_load_round(p.pe, c.s, min(c.e - c.s, kPcRound), lane, R);
                int4 W[4] = {};
                if (ALGO == ALG_SSSP) {
                    uint4 Wu[4];
                    pc_load_round(reinterpret_cast<const uint32_t *>(p.pw), cs, cn, lane, Wu);
#pragma unroll
                    for (int q = 0; q < 4; ++q) W[q] = make_int4((int)Wu[q].x, (int)Wu[q].y, (int)Wu[q].z, (int)Wu[q].w);
                }
                // NULL messages need a test only where NULL is not the monoid identity
                constexpr bool kNul = ALGO == ALG_SSSP || ALGO == ALG_PPR || ALGO == ALG_NIBBLE;
                if (ALGO == ALG_PR && chk) {
                    if (cn <= 128) pc_round<ALGO, B16, 4, true>(E, W, cn, vals, acc_o, lane);
                    else if (cn <= 256) pc_round<ALGO, B16, 8, true>(E, W, cn, vals, acc_o, lane);
                    else pc_round<ALGO, B16, 16, true>(E, W, cn, vals, acc_o, lane);
                } else {
                    if (cn <= 128) pc_round<ALGO, B16, 4, kNul>(E, W, cn, vals, acc_o, lane);
                    else if (cn <= 256) pc_round<ALGO, B16, 8, kNul>(E, W, cn, vals, acc_o, lane);
                    else pc_round<ALGO, B16, 16, kNul>(E, W, cn, vals, acc_o, lane);
                }
            }
            // the buffer is released only after its values were waited for and read: after an abort it is
            // not, so that the producer never re-arms a buffer whose copy may still be in flight.  Warps own
            // the same destinations in every block of the task, so they need not wait for one another here.
            __syncwarp();
            if (ok && lane == 0) mbar_arrive(&empty[b]);
        }
        if (pc_consumers_or(!ok)) break;  // an abort: all consumers leave together
        // the column's result, or this task's partial vector of a column split over several tasks; the
        // accumulator is reset as it is read (each word by the thread that reads it)
        const uint4 tk = sl.tk;
        const uint32_t gq = tk.x << p.shift, wq = min(p.P, p.V - gq);
        uint32_t *out = (tk.w == kNull) ? p.pc_sum + gq : p.pc_part + (uint64_t)tk.w * p.P;
        for (uint32_t i = threadIdx.x; i < wq; i += kPcGatherWarps * 32) {
            const uint32_t a = pc_swz(i);
            out[i] = acc[a];
            acc[a] = O::identity();
        }
        pc_consumers_sync();
        if (lane == 0) mbar_arrive(&tempty[ts]);
    }
}

// PC part of the gather (Alg. 2 gather over the PC bins, Sec. 3.1.2): one CTA per SM takes tasks (ranges of
// consecutive blocks of one column's message sequence) with a producer warp and kPcGatherWarps consumer warps.
//  * The producer stages each active block's message values in one of nbuf shared buffers (TMA bulk copies
//    of its bin runs), up to nbuf blocks ahead of the slowest consumer; "full" / "empty" mbarriers per
//    buffer replace a CTA barrier per block, so consumer warps drift within that window.
//  * Consumer warp w folds the w-th destination slice of every block through the prestored destination
//    entries (loaded straight from global memory into registers, one round ahead) into the shared column
//    accumulator, with lane-serial runs and a segmented warp scan: random accesses touch shared memory
//    only, and no atomics are used, so sums are taken in a fixed order.
// The accumulator stays in shared memory for the whole task (at swizzled positions); a column split over
// several tasks writes one partial vector per task.  Every mbarrier wait is bounded: when one runs out,
// the run's error flag is raised and all warps leave, the producer after its copies have landed.
template <int ALGO, bool B16>
__global__ void __launch_bounds__(kPcThreads, 1) k_gather_pc(Params p) {
    using O = Op<ALGO>;
    constexpr uint32_t kStageWords = kPcBlock + 4;
    extern __shared__ __align__(16) uint32_t s_pc_dyn[];
    const uint32_t nbuf = p.pc_nbuf;
    uint32_t *stage = s_pc_dyn;                     // nbuf x (kPcBlock message values, the padding slot, a scratch word)
    uint32_t *acc = s_pc_dyn + nbuf * kStageWords;  // P values of the column
    __shared__ __align__(8) uint64_t s_full[kPcMaxBufs], s_empty[kPcMaxBufs], s_tfull[2], s_tempty[2];
    __shared__ PcSlot s_slot[2];
    __shared__ uint32_t s_abort;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < nbuf; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], kPcGatherWarps);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&s_tfull[i], 1);
            mbar_init(&s_tempty[i], kPcGatherWarps);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    // value slot of the padding entries (the copies never write it): the monoid identity, so padding folds
    // as a no-op whether or not NULLs are checked.  BF16 only carries sums: its identity is +0.
    if (threadIdx.x < nbuf) {
        if (B16) reinterpret_cast<uint16_t *>(stage + threadIdx.x * kStageWords)[kPcPadIdx] = 0;
        else stage[threadIdx.x * kStageWords + kPcPadIdx] = O::identity();
    }
    for (uint32_t i = threadIdx.x; i < p.P; i += kPcThreads) acc[i] = O::identity();
    // the set-up above touches shared memory only, so it overlaps the end of the scatter; from here on
    // the scatter's messages and the plan's counters are read
    GPOP_GRID_DEP();
    const unsigned long long t_start = p.t_gpc ? globaltimer() : 0ull;
    __syncthreads();
    if (wid == kPcGatherWarps)
        pc_producer<B16>(p, s_slot, s_full, s_empty, s_tfull, s_tempty, stage, nbuf, &s_abort, lane);
    else
        pc_consumer<ALGO, B16>(p, s_slot, s_full, s_empty, s_tfull, s_tempty, stage, acc, nbuf, &s_abort,
                               lane, wid);
    if (p.t_gpc && threadIdx.x == 0) atomicAdd(p.t_gpc, globaltimer() - t_start);
}

// Result of the PC gather for the columns split over several k_gather_pc tasks: each 1024-destination
// chunk of such a column combines the column's partial vectors in task order (a fixed order, so sums are
// reproducible) into pc_sum; one chunk per CTA, 16-byte accesses.
template <int ALGO>
__global__ void __launch_bounds__(256) k_merge_pc(Params p) {
    GPOP_GRID_DEP();
    using O = Op<ALGO>;
    for (uint32_t it = blockIdx.x; it < p.nmerge; it += gridDim.x) {
        const uint2 m = p.pc_merge[it];  // column, first destination
        if (p.gflag_pc[m.x] != p.epoch) continue;
        const uint32_t gq = m.x << p.shift, wq = min(p.P, p.V - gq);
        const uint32_t nt = p.col_ntask[m.x], part0 = p.col_part0[m.x];
        const uint32_t i = m.y + threadIdx.x * 4;
        if (i >= min(wq, m.y + 1024)) continue;
        const uint32_t *src = p.pc_part + (uint64_t)part0 * p.P + i;
        if (i + 4 <= wq) {
            uint4 r = make_uint4(O::identity(), O::identity(), O::identity(), O::identity());
            // eight partial vectors' loads in flight, combined in task order
            for (uint32_t j0 = 0; j0 < nt; j0 += 8) {
                uint4 v[8];
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u)
                    v[u] = j0 + u < nt ? __ldcs(reinterpret_cast<const uint4 *>(src + (uint64_t)(j0 + u) * p.P))
                                       : make_uint4(0, 0, 0, 0);
#pragma unroll
                for (uint32_t u = 0; u < 8; ++u)
                    if (j0 + u < nt)
                        r = make_uint4(O::combine(r.x, v[u].x), O::combine(r.y, v[u].y), O::combine(r.z, v[u].z),
                                       O::combine(r.w, v[u].w));
            }
            *reinterpret_cast<uint4 *>(p.pc_sum + gq + i) = r;
        } else {
            for (uint32_t c = i; c < wq; ++c) {
                uint32_t r = O::identity();
                for (uint32_t j = 0; j < nt; ++j) r = O::combine(r, src[(uint64_t)j * p.P + (c - i)]);
                p.pc_sum[gq + c] = r;
            }
        }
    }
}

// Task accumulator of the SC pass: a 32-bit word per destination for the min / AND monoids, and for the
// sums (PR, PPR, Nibble, whose values are probability masses: every sum lies in [0, 1]) an unsigned
// 64-bit fixed-point number with 62 fraction bits.  A message converts exactly when it is at least 2^-39
// (within 2^-63 below that), the integer additions are exact and independent of the order in which the
// pairs arrive (a hub destination can receive very many), and the filter rounds the total to FP32 once.
// 64-bit integer atomics are native on shared memory; FP64 ones are not, and FP64 is scarce on this GPU.
constexpr float kFixOne = 0x1p62f;    // 2^62
constexpr float kFixUnit = 0x1p-62f;  // 2^-62
template <int ALGO>
struct ScAcc {
    static constexpr bool kSum = sums(ALGO);
    using T = typename std::conditional<kSum, unsigned long long, uint32_t>::type;
    static __device__ __forceinline__ T from_msg(uint32_t m) {
        if constexpr (kSum) return __float2ull_rn(u2f(m) * kFixOne);
        else return m;
    }
    static __device__ __forceinline__ uint32_t to_msg(T a) {
        if constexpr (kSum) return f2u(__ull2float_rn(a) * kFixUnit);
        else return a;
    }
    // folds one SC pair's value v into acc[d]: atomic minimum (BFS parents, CC labels, SSSP distances), AND
    // (multi-source BFS) or fixed-point addition, none of whose results depends on the order of the pairs
    static __device__ __forceinline__ void fold(T *acc, uint32_t d, uint32_t v) {
        if constexpr (kSum) atomicAdd(&acc[d], from_msg(v));
        else if constexpr (ALGO == ALG_MSBFS) atomicAnd(&acc[d], v);
        else atomicMin(&acc[d], v);
    }
};

// Gather of one (column q, destination range) task, after k_gather_pc:
//  1. PC messages: the column's PC result (pc_sum), only when some partition sent PC messages to the
//     column this iteration;
//  2. SC pairs of the task's fresh SC bins, folded with shared atomics;
//  3. reInit / gather apply / filter of every destination of the range and the next frontier (Alg. 2).
// SC pair j of a bin region: (local destination, message value bits), 8 bytes, or 4 bytes with BF16 values
template <bool B16>
__device__ __forceinline__ uint2 sc_pair(const Params &p, uint32_t j) {
    if (B16) {
        const uint32_t w = reinterpret_cast<const uint32_t *>(p.scpair)[j];
        return make_uint2(w & 0xFFFFu, from_bf16(w >> 16));
    }
    return p.scpair[j];
}

template <int ALGO, bool B16>
__global__ void __launch_bounds__(kGatherThreads) k_gather(Params p) {
    GPOP_GRID_DEP();
    using O = Op<ALGO>;
    using A = ScAcc<ALGO>;
    __shared__ typename A::T s_acc[kGatherWidth];
    __shared__ uint32_t s_task, s_next, s_nbig, s_big[kMaxBigScBins], s_last;
    __shared__ uint32_t s_va[kGatherWarps];
    __shared__ unsigned long long s_ea[kGatherWarps];
    __shared__ double s_res[kGatherWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    for (;;) {
        if (tid == 0) s_task = atomicAdd(&p.counters[2], 1u);
        __syncthreads();
        const uint32_t t = s_task;
        __syncthreads();
        if (t >= p.ngt) break;
        const GatherTask gt = p.gtask[t];
        const uint32_t q = gt.q;
        if (p.gflag[q] != p.epoch) continue;
        unsigned long long t0 = (p.t_task && tid == 0) ? globaltimer() : 0ull;
        const uint32_t width = gt.d1 - gt.d0;
        const uint32_t gq = q << p.shift;
        const uint32_t gbase = gq + gt.d0;
        const uint32_t wv = min(width, p.V - gbase);  // destinations that exist
        if (tid == 0 && p.gath) atomicAdd(p.gath, (unsigned long long)wv);
        // the column's PC result (pc_sum: written by its k_gather_pc task, or merged by k_merge_pc from the
        // partial vectors of a split column); none when no partition sent PC messages to the column this
        // iteration or the column has no PC in-edges.  Without SC pairs the filter reads it directly.
        const bool has_pc = p.gflag_pc[q] == p.epoch && p.col_ntask[q] > 0;
        const uint32_t nfresh = p.task_sc_cnt[t];
        const bool direct = nfresh == 0;
        if (!direct) {
            for (uint32_t i = tid; i < width; i += nthr)
                s_acc[i] = A::from_msg((has_pc && i < wv) ? p.pc_sum[gbase + i] : O::identity());
            __syncthreads();
        }

        // SC messages: the task's fresh SC bins (binPartList) are dealt to the warps dynamically, a
        // lane per pair, each pair folded into the accumulator with one shared atomic (min for BFS /
        // CC / SSSP, float add for PR / PPR); bins of at least kBigScBin pairs are left to a second,
        // CTA-wide pass so that no single warp carries a hub partition's bin alone
        if (nfresh) {
            const unsigned long long tsc0 = (p.t_gsc && tid == 0) ? globaltimer() : 0ull;
            const uint32_t lbase = p.task_sub_ptr[t];
            if (tid == 0) {
                s_next = 0;
                s_nbig = 0;
            }
            __syncthreads();
            for (;;) {
                uint32_t i = 0;
                if (lane == 0) i = atomicAdd(&s_next, 1u);
                i = __shfl_sync(0xffffffffu, i, 0);
                if (i >= nfresh) break;
                const uint32_t bn = p.task_sc_list[lbase + i];
                const uint32_t cnt = p.sccnt[bn], sb = p.sub_cap[bn];
                if (cnt >= kBigScBin) {
                    uint32_t k = 0;
                    if (lane == 0) k = atomicAdd(&s_nbig, 1u);
                    k = __shfl_sync(0xffffffffu, k, 0);
                    if (k < kMaxBigScBins) {
                        if (lane == 0) s_big[k] = bn;
                        continue;
                    }
                }
                for (uint32_t j = lane; j < cnt; j += 32) {
                    const uint2 pr = sc_pair<B16>(p, sb + j);
                    A::fold(s_acc, pr.x - gt.d0, pr.y);
                }
            }
            __syncthreads();
            const uint32_t nbig = min(s_nbig, kMaxBigScBins);
            for (uint32_t k = 0; k < nbig; ++k) {
                const uint32_t bn = s_big[k];
                const uint32_t cnt = p.sccnt[bn], sb = p.sub_cap[bn];
                for (uint32_t j = tid; j < cnt; j += nthr) {
                    const uint2 pr = sc_pair<B16>(p, sb + j);
                    A::fold(s_acc, pr.x - gt.d0, pr.y);
                }
            }
            __syncthreads();
            if (p.t_gsc && tid == 0) atomicAdd(p.t_gsc, globaltimer() - tsc0);
        }

        // reInit (init of previously active vertices), gather apply, filter, next frontier.
        // Each thread takes 4 consecutive destinations (16-byte vector accesses); 8 threads form
        // one 32-bit frontier word.
        uint32_t va = 0;
        unsigned long long ea = 0;
        double res = 0.0;
        const uint32_t wround = (width + 31) & ~31u;
        // the bound is tested on the warp's first destination so that every lane of a warp runs the
        // same iterations (the word assembly below uses full-warp shuffles)
        for (uint32_t i0 = tid * 4; i0 - (uint32_t)lane * 4 < wround; i0 += nthr * 4) {
            const uint32_t g0 = gbase + i0;
            const bool any = i0 < wv;
            uint32_t nib = 0;
            uint32_t fresh[4] = {0u, 0u, 0u, 0u};  // multi-source BFS: sources reaching each vertex first now
            uint32_t was_word = any ? p.bits[g0 >> 5] : 0u;
            if (any) {
                const bool full = i0 + 4 <= wv;
                uint4 rp = full ? *reinterpret_cast<const uint4 *>(p.rowptr + g0) : make_uint4(0, 0, 0, 0);
                uint32_t rp4 = p.rowptr[min(g0 + 4, p.V)];
                uint32_t rpv[5] = {rp.x, rp.y, rp.z, rp.w, rp4};
                if (!full)
                    for (int c = 0; c < 4; ++c) rpv[c] = (i0 + c < wv) ? p.rowptr[g0 + c] : rp4;
                uint4 vv = full ? *reinterpret_cast<const uint4 *>(p.val + g0) : make_uint4(0, 0, 0, 0);
                uint32_t vals[4] = {vv.x, vv.y, vv.z, vv.w};
                uint32_t lv[4] = {kInf, kInf, kInf, kInf};
                if (!full)
                    for (int c = 0; c < 4; ++c) vals[c] = (i0 + c < wv) ? p.val[g0 + c] : 0u;
                uint32_t msg[4] = {O::identity(), O::identity(), O::identity(), O::identity()};
                if (!direct) {
                    for (int c = 0; c < 4; ++c) msg[c] = A::to_msg(s_acc[min(i0 + c, width - 1)]);
                } else if (has_pc) {
                    if (full) {
                        const uint4 m4 = *reinterpret_cast<const uint4 *>(p.pc_sum + g0);
                        msg[0] = m4.x; msg[1] = m4.y; msg[2] = m4.z; msg[3] = m4.w;
                    } else {
                        for (int c = 0; c < 4; ++c) msg[c] = (i0 + c < wv) ? p.pc_sum[g0 + c] : O::identity();
                    }
                }
                if (ALGO == ALG_BFS) {
                    if (full) {
                        uint4 l4 = *reinterpret_cast<const uint4 *>(p.lvl + g0);
                        lv[0] = l4.x; lv[1] = l4.y; lv[2] = l4.z; lv[3] = l4.w;
                    } else {
                        for (int c = 0; c < 4; ++c) lv[c] = (i0 + c < wv) ? p.lvl[g0 + c] : 0u;
                    }
                }
                uint32_t nv[4], ns[4];
                bool wrote_lv = false;
                // L1 change of the four vertices: each |x_new - x_old| rounded once in FP32 and their sum
                // carried in FP64 (FP64 instructions are scarce on this GPU: one conversion and one add
                // per four vertices)
                float res4 = 0.f;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t g = g0 + c;
                    nv[c] = vals[c];
                    ns[c] = kNull;
                    if (i0 + c >= wv) continue;
                    const bool was = (was_word >> (g & 31)) & 1u;
                    const uint32_t m = msg[c];
                    const uint32_t deg = rpv[c + 1] - rpv[c];
                    bool act = false;
                    if (ALGO == ALG_PR) {
                        // Alg. 6: initFunc PR = 0 (continue), gatherFunc +=, filterFunc damping
                        float xo = u2f(vals[c]);
                        float xn = fmaf(p.c1, u2f(m), p.c0);
                        nv[c] = f2u(xn);
                        res4 += fabsf(xn - xo);
                        act = true;
                        ns[c] = f2u(deg ? xn / (float)deg : 0.f);
                    } else if (ALGO == ALG_PPR) {
                        // initFunc PR = 0, continue iff seed; gatherFunc +=; filterFunc restart, keep iff > 0
                        float xo = u2f(vals[c]);
                        bool cont = was && g == p.source;
                        bool recv = m != 0u;
                        float xn = 0.f;
                        if (cont || recv) xn = fmaf(p.c1, u2f(m), g == p.source ? p.c0 : 0.f);
                        act = (cont || recv) && xn > 0.f;
                        nv[c] = f2u(xn);
                        res4 += fabsf(xn - xo);
                        if (act) ns[c] = f2u(deg ? xn / (float)deg : 0.f);
                    } else if (ALGO == ALG_NIBBLE) {
                        // Alg. 4: initFunc halves PR of a frontier vertex (update1) and keeps it on iff
                        // PR >= eps deg (cond1); gatherFunc adds the messages and activates the vertex;
                        // filterFunc keeps it iff PR >= eps deg (cond2).  A sink never stays on.
                        const float xo = u2f(vals[c]);
                        const float thr = p.eps * (float)deg;
                        float x = xo;
                        bool keep = false;
                        if (was) {
                            x = 0.5f * x;
                            keep = deg > 0 && x >= thr;
                        }
                        const bool recv = m != 0u;
                        if (recv) x = x + u2f(m);
                        act = (keep || recv) && deg > 0 && x >= thr;
                        nv[c] = f2u(x);
                        res4 += fabsf(x - xo);
                        if (act) ns[c] = f2u(x / (2.f * (float)deg));
                    } else if (ALGO == ALG_MSBFS) {
                        // Alg. 5 for every source of the pass at once: the sources that reach the vertex
                        // (complement of the AND of complemented sets) minus those that already had it
                        const uint32_t nw = ~m & ~vals[c];
                        if (nw) {
                            fresh[c] = nw;
                            nv[c] = vals[c] | nw;
                            act = true;
                            ns[c] = ~nw;
                        }
                    } else if (ALGO == ALG_BFS) {
                        // Alg. 5: first discovery sets the parent (smallest candidate) and level
                        if (m != kInf && lv[c] == kInf) {
                            lv[c] = p.iter;
                            wrote_lv = true;
                            nv[c] = m;
                            act = true;
                            ns[c] = g;
                        }
                    } else {
                        // Alg. 7 / CC: keep the minimum distance or label, activate on improvement; with
                        // interleaved scatter-gather, an active vertex whose partition was not in this
                        // iteration's wave stays active (it has not scattered yet)
                        if (m < vals[c]) {
                            nv[c] = m;
                            act = true;
                            ns[c] = m;
                        } else if (p.isg_w >= 2 && was && q % p.isg_w != (p.iter - 1) % p.isg_w) {
                            act = true;
                            ns[c] = vals[c];
                        }
                    }
                    if (act) {
                        nib |= 1u << c;
                        va++;
                        ea += deg;
                    }
                }
                if (sums(ALGO)) res += (double)res4;
                if (full) {
                    if (nv[0] != vals[0] || nv[1] != vals[1] || nv[2] != vals[2] || nv[3] != vals[3])
                        *reinterpret_cast<uint4 *>(p.val + g0) = make_uint4(nv[0], nv[1], nv[2], nv[3]);
                    *reinterpret_cast<uint4 *>(p.sval + g0) = make_uint4(ns[0], ns[1], ns[2], ns[3]);
                    if (ALGO == ALG_BFS && wrote_lv)
                        *reinterpret_cast<uint4 *>(p.lvl + g0) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                } else {
                    for (int c = 0; c < 4; ++c)
                        if (i0 + c < wv) {
                            if (nv[c] != vals[c]) p.val[g0 + c] = nv[c];
                            p.sval[g0 + c] = ns[c];
                            if (ALGO == ALG_BFS) p.lvl[g0 + c] = lv[c];
                        }
                }
            }
            if (ALGO == ALG_MSBFS) {
                // level rows: the warp walks the sources any of its lanes reached, so that the stores to
                // one row come from consecutive lanes
                const uint32_t mine = fresh[0] | fresh[1] | fresh[2] | fresh[3];
                uint32_t wall = __reduce_or_sync(0xffffffffu, mine);
                while (wall) {
                    const int j = __ffs(wall) - 1;
                    wall &= wall - 1;
                    if ((mine >> j) & 1u) {
                        uint32_t *row = p.lvl_ms + (uint64_t)j * p.V + g0;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if ((fresh[c] >> j) & 1u) row[c] = p.iter;
                    }
                }
            }
            // 8 consecutive threads own one frontier word
            uint32_t word = nib << (i0 & 31);
            word |= __shfl_xor_sync(0xffffffffu, word, 1);
            word |= __shfl_xor_sync(0xffffffffu, word, 2);
            word |= __shfl_xor_sync(0xffffffffu, word, 4);
            if ((lane & 7) == 0 && i0 < wround && (gbase + (i0 & ~31u)) < p.V)
                p.bits[(gbase + (i0 & ~31u)) >> 5] = word;
        }
        for (int o = 16; o > 0; o >>= 1) {
            va += __shfl_xor_sync(0xffffffffu, va, o);
            ea += __shfl_xor_sync(0xffffffffu, ea, o);
            res += __shfl_xor_sync(0xffffffffu, res, o);
        }
        if (lane == 0) { s_va[wid] = va; s_ea[wid] = ea; s_res[wid] = res; }
        __syncthreads();
        if (tid == 0) {
            uint32_t a = 0;
            unsigned long long b2 = 0;
            double r = 0.0;
            for (int w = 0; w < kGatherWarps; ++w) { a += s_va[w]; b2 += s_ea[w]; r += s_res[w]; }
            p.t_va[t] = a;
            p.t_ea[t] = b2;
            p.t_res[t] = __double2ull_rn(r * kResOne);
            p.t_stamp[t] = p.epoch;
            if (p.t_task) p.t_task[t] = globaltimer() - t0;
            s_last = 0;
            if (p.col_done) {  // learned policy: the column's last task to finish picks its next mode
                __threadfence();
                s_last = atomicAdd(&p.col_done[q], 1u) == p.col_task[q + 1] - p.col_task[q] - 1;
            }
        }
        __syncthreads();
        if (s_last && wid == 0) {
            __threadfence();
            select_partition(p, q, p.epoch, lane);
            if (lane == 0) p.col_done[q] = 0;
        }
    }
}

// --- host side --------------------------------------------------------------------------------

struct RunBuffers {
    uint32_t *val = nullptr, *lvl = nullptr, *sval = nullptr, *bits = nullptr;
    uint32_t *t_va = nullptr, *t_stamp = nullptr;
    unsigned long long *t_ea = nullptr;
    unsigned long long *t_res = nullptr;
    uint8_t *mode = nullptr, *action = nullptr, *sel_mode = nullptr;
    uint32_t *col_done = nullptr;
    uint32_t *gflag = nullptr, *gflag_pc = nullptr, *counters = nullptr;
    uint4 *sc_list = nullptr;
    uint32_t *sc_gcur = nullptr, *sc_udone = nullptr, *pc_prefix = nullptr, *sc_seg = nullptr;
    uint32_t *task_sc_cnt = nullptr, *task_sc_list = nullptr, *pc_sum = nullptr;
    unsigned long long *gath = nullptr;  // destinations visited by k_gather in the current run
    Control *ctrl = nullptr, *h_ctrl = nullptr, *d_ctrl_snap = nullptr;
    // LOG_BOTH only (allocated on first use)
    uint32_t *shadow = nullptr, *part_va = nullptr;
    uint4 *all_list = nullptr;
    unsigned long long *part_ea = nullptr, *t_pc = nullptr, *t_sc = nullptr, *t_gpc = nullptr, *t_gsc = nullptr;
    double rate_pc = 0.0, rate_sc = 0.0;  // LOG_BOTH: gather ns per modelled byte, last measured per mode
    float *feat = nullptr;
    // multi-source BFS (allocated on first use): the pass's sources, staged level rows for host output
    uint32_t *msrc = nullptr, *lvl_ms = nullptr;
    // the state the last successful run left (val, lvl, sval, bits), for gpop_state_export and resume:
    // its algorithm (-1: none), the iterations behind it and the L1 change of its last gather
    int state_algo = -1;
    uint32_t state_iter = 0;
    double state_res = 0.0;
    // the options of that run that shape its result (a resumed run must repeat them)
    uint32_t state_source = 0, state_bf16 = 0;
    double state_damping = 0.0, state_epsilon = 0.0;
};

static void release_runbufs(RunBuffers *rb) {
    void *ptrs[] = {rb->val, rb->lvl, rb->sval, rb->bits, rb->t_va, rb->t_stamp, rb->t_ea, rb->t_res,
                    rb->mode, rb->action, rb->sel_mode, rb->col_done, rb->gflag, rb->gflag_pc, rb->sc_list, rb->sc_gcur, rb->sc_udone, rb->pc_prefix, rb->sc_seg, rb->counters,
                    rb->ctrl, rb->task_sc_cnt, rb->task_sc_list, rb->pc_sum, rb->gath, rb->shadow, rb->all_list, rb->part_va, rb->part_ea, rb->t_pc, rb->t_sc, rb->t_gpc, rb->t_gsc,
                    rb->feat, rb->msrc, rb->lvl_ms};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (rb->h_ctrl) cudaFreeHost(rb->h_ctrl);
    delete rb;
}

// SC scatter units of one iteration: one per SC partition plus one per kScUnitEdges active edges
static uint64_t sc_unit_capacity(const Graph *g) { return (uint64_t)g->k + g->E / kScUnitEdges + 2; }

static gpop_status alloc_runbufs(Graph *g, RunBuffers **out) {
    RunBuffers *rb = new RunBuffers();
    uint64_t nw = (g->V + 31) / 32 + 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **ptr, uint64_t n) {
        if (e == cudaSuccess) e = dalloc(g, ptr, n);
    };
    A(&rb->val, g->V);
    A(&rb->lvl, g->V);
    A(&rb->sval, g->V);
    A(&rb->bits, nw);
    A(&rb->t_va, g->ngt);
    A(&rb->t_stamp, g->ngt);
    A(&rb->t_ea, g->ngt);
    A(&rb->t_res, g->ngt);
    A(&rb->mode, g->k);
    A(&rb->action, g->k);
    A(&rb->sel_mode, g->k);
    A(&rb->col_done, g->k);
    A(&rb->gflag, g->k);
    A(&rb->gflag_pc, g->k);
    A(&rb->sc_list, sc_unit_capacity(g));
    A(&rb->sc_gcur, std::max<uint64_t>(g->nsub, 1));
    A(&rb->sc_seg, (uint64_t)g->k * kScSegs);
    A(&rb->sc_udone, g->k);
    A(&rb->pc_prefix, (uint64_t)g->k + 1);
    A(&rb->counters, 8);
    A(&rb->task_sc_cnt, g->ngt);
    A(&rb->pc_sum, g->V);
    A(&rb->gath, 1);
    A(&rb->task_sc_list, g->nsub);
    A(&rb->ctrl, 1);
    // the plans' snapshots: two slots of mapped pinned memory that k_plan writes directly (no copy in the
    // stream between a plan and its iteration's kernels)
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&rb->h_ctrl, 2 * sizeof(Control), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&rb->d_ctrl_snap, rb->h_ctrl, 0);
    if (e == cudaSuccess) e = cudaMemset(rb->t_stamp, 0, 4ull * std::max<uint32_t>(g->ngt, 1));
    if (e == cudaSuccess) e = cudaMemset(rb->gflag, 0, 4ull * g->k);
    if (e == cudaSuccess) e = cudaMemset(rb->gflag_pc, 0, 4ull * g->k);
    if (e == cudaSuccess) e = cudaMemset(rb->task_sc_cnt, 0, 4ull * std::max<uint32_t>(g->ngt, 1));
    if (e == cudaSuccess) e = cudaMemset(rb->bits, 0, 4ull * nw);
    if (e == cudaSuccess) e = cudaMemset(rb->sc_gcur, 0, 4ull * std::max<uint64_t>(g->nsub, 1));
    if (e == cudaSuccess) e = cudaMemset(rb->sc_udone, 0, 4ull * g->k);
    if (e == cudaSuccess) e = cudaMemset(rb->col_done, 0, 4ull * g->k);
    if (e != cudaSuccess) {
        release_runbufs(rb);
        return fail(e == cudaErrorMemoryAllocation ? GPOP_ERR_OOM : GPOP_ERR_CUDA,
                    std::string("run buffers: ") + cudaGetErrorString(e));
    }
    *out = rb;
    return GPOP_OK;
}

void release_run_state(Graph *g) {
    if (g->run) release_runbufs(static_cast<RunBuffers *>(g->run));
    g->run = nullptr;
}

template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int num_sms) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    return std::max(1, per) * num_sms;
}

// LOG_BOTH: turns this iteration's per-task CTA durations into one record per scattered partition:
// 8 features, t_PC and t_SC in microseconds (the partition's share of that mode's shadow scatter wall
// time, in proportion to its CTA time there, + that mode's share of the gather, attributed by gather bytes
// at the iteration's measured gather SM time per byte), the mode Eq. (mode) chose, the partition and the
// iteration.  occ: resident CTAs per SM of k_scatter_pc, k_scatter_sc and k_gather; ev: events before the
// shadow PC scatter, between the shadows and after the shadow SC scatter.
static gpop_status log_iteration(Graph *g, RunBuffers *rb, const gpop_run_opts *o, cudaStream_t s, uint32_t iter,
                                 gpop_run_stats *st, const double occ[3], cudaEvent_t const ev[3]) {
    const uint32_t k = g->k;
    std::vector<float> feat(8ull * k);
    std::vector<uint32_t> va(k);
    std::vector<unsigned long long> ea(k), tpc(g->nst), tsc(k), tgpc(1, 0), tgsc(1, 0);
    std::vector<uint8_t> mode(k);
    std::vector<ScatterTask> stask(g->nst);
    GPOP_CUDA_TRY(cudaMemcpyAsync(feat.data(), rb->feat, 4ull * 8 * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(va.data(), rb->part_va, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(ea.data(), rb->part_ea, 8ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(mode.data(), rb->mode, k, cudaMemcpyDeviceToHost, s));
    if (g->nst) {
        GPOP_CUDA_TRY(cudaMemcpyAsync(tpc.data(), rb->t_pc, 8ull * g->nst, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaMemcpyAsync(stask.data(), g->stask, sizeof(ScatterTask) * g->nst, cudaMemcpyDeviceToHost, s));
    }
    GPOP_CUDA_TRY(cudaMemcpyAsync(tsc.data(), rb->t_sc, 8ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(tgpc.data(), rb->t_gpc, 8, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(tgsc.data(), rb->t_gsc, 8, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<double> pc_ns(k, 0.0);
    for (uint32_t t = 0; t < g->nst; ++t)
        if (mode[stask[t].p] != kModeNone) pc_ns[stask[t].p] += (double)tpc[t];
    // each shadow scatter's wall time (CUDA events around it), shared among the partitions in proportion to
    // their CTA times: the scatter part of a label then adds up to that mode's measured wall time
    float w_pc_ms = 0.f, w_sc_ms = 0.f;
    GPOP_CUDA_TRY(cudaEventElapsedTime(&w_pc_ms, ev[0], ev[1]));
    GPOP_CUDA_TRY(cudaEventElapsedTime(&w_sc_ms, ev[1], ev[2]));
    double sum_pc = 0.0, sum_sc = 0.0;
    for (uint32_t q = 0; q < k; ++q)
        if (mode[q] != kModeNone) {
            sum_pc += pc_ns[q];
            sum_sc += (double)tsc[q];
        }
    const double f_pc = sum_pc > 0 ? 1e6 * w_pc_ms / sum_pc : 1.0 / occ[0];
    const double f_sc = sum_sc > 0 ? 1e6 * w_sc_ms / sum_sc : 1.0 / occ[1];
    // gather time per mode, attributed to the partitions of that mode by the bytes their messages make
    // the gather read (PC: 4 B per message value + 4 B per destination entry, folded by k_gather_pc; SC:
    // 8 B per pair, folded by k_gather's SC pass); the mode Eq. (mode) did not pick is charged at the last
    // rate measured for it in this run (the other mode's rate until one is)
    auto gb = [&](uint32_t q, int m) {
        return m == kModePC ? 4.0 * (double)g->h_npng[q] + 4.0 * (double)g->h_Ep[q] : 8.0 * (double)ea[q];
    };
    double bytes_pc = 0.0, bytes_sc = 0.0;
    for (uint32_t q = 0; q < k; ++q) {
        if (mode[q] == kModePC) bytes_pc += gb(q, kModePC);
        if (mode[q] == kModeSC) bytes_sc += gb(q, kModeSC);
    }
    // CTA times become SM times (divided by the kernel's resident CTAs per SM: k_gather_pc has one per SM,
    // the SC scatter and the task gather several), so that both modes are charged in the unit that adds up
    // to wall time on a full GPU
    if (bytes_pc > 0) rb->rate_pc = (double)tgpc[0] / bytes_pc;
    if (bytes_sc > 0) rb->rate_sc = (double)tgsc[0] / occ[2] / bytes_sc;
    const double rpc = rb->rate_pc > 0 ? rb->rate_pc : rb->rate_sc, rsc = rb->rate_sc > 0 ? rb->rate_sc : rb->rate_pc;
    for (uint32_t q = 0; q < k; ++q) {
        if (mode[q] == kModeNone || st->log_records >= o->log_capacity) continue;
        float *r = o->log_buffer + st->log_records * GPOP_LOG_RECORD_FLOATS;
        for (int i = 0; i < 8; ++i) r[i] = feat[8ull * q + i];
        r[8] = (float)((pc_ns[q] * f_pc + rpc * gb(q, kModePC)) / 1e3);
        r[9] = (float)(((double)tsc[q] * f_sc + rsc * gb(q, kModeSC)) / 1e3);
        r[10] = (float)mode[q];
        r[11] = (float)q;
        r[12] = (float)iter;
        st->log_records++;
    }
    (void)va;
    return GPOP_OK;
}

// One pass of a multi-source BFS: device array of n <= 32 sources and the device level rows (n x V words)
struct MsPass {
    const uint32_t *src;
    uint32_t n;
    uint32_t *lvl;
};

template <int ALGO, bool B16>
static gpop_status run_algo(Graph *g, RunBuffers *rb, const gpop_run_opts *o, cudaStream_t s, void *out_values,
                            uint32_t *out_parent, int out_is_device, gpop_run_stats *stats,
                            const MsPass *mpass = nullptr) {
    Params p{};  // every field starts at zero / null
    memset(&p, 0, sizeof p);
    p.V = g->V; p.P = g->P; p.shift = g->shift; p.k = g->k;
    p.rowptr = g->rowptr; p.col = g->col; p.w = g->w; p.esub = g->esub;
    p.row_bin = g->row_bin; p.bin_q = g->bin_q; p.col_bin = g->col_bin; p.col_bins = g->col_bins;
    p.png = g->png; p.pdata = g->pdata; p.row_png = g->row_png;
    p.pc_runs = g->pc_runs; p.pc_task = g->pc_task; p.pc_wsp = g->pc_wsp; p.pc_tsp = g->pc_tsp; p.pc_blk_run = g->pc_blk_run; p.pc_blk_nval = g->pc_blk_nval; p.pc_blk_prange = g->pc_blk_prange; p.pc_merge = g->pc_merge; p.nmerge = g->nmerge; p.pc_blk_ent = g->pc_blk_ent;
    p.scpair = g->scpair; p.sccnt = g->sccnt;
    p.sub_cap = g->sub_cap; p.sub_task = g->sub_task; p.row_sub = g->row_sub; p.task_sub_ptr = g->task_sub_ptr;
    p.task_sc_cnt = rb->task_sc_cnt; p.task_sc_list = rb->task_sc_list;
    p.col_ntask = g->col_ntask; p.col_part0 = g->col_part0; p.pe = g->pe; p.pw = g->pw; p.pc_part = g->pc_part;
    p.npct = g->npct; p.pc_sum = rb->pc_sum; p.gath = rb->gath;
    p.Ep = g->Ep; p.npng_p = g->npng_p;
    p.gtask = g->gtask; p.ngt = g->ngt; p.col_task = g->col_task;
    p.stask = g->stask; p.nst = g->nst; p.pc_state = g->pc_state;
    p.val = rb->val; p.lvl = rb->lvl; p.sval = rb->sval; p.bits = rb->bits;
    p.t_va = rb->t_va; p.t_ea = rb->t_ea; p.t_res = rb->t_res; p.t_stamp = rb->t_stamp;
    p.mode = rb->mode; p.action = rb->action; p.sel_mode = rb->sel_mode; p.gflag = rb->gflag; p.gflag_pc = rb->gflag_pc;
    p.sc_list = rb->sc_list; p.sc_seg = rb->sc_seg; p.sc_gcur = rb->sc_gcur; p.sc_udone = rb->sc_udone; p.pc_prefix = rb->pc_prefix; p.counters = rb->counters; p.ctrl = rb->ctrl; p.ctrl_snap = rb->d_ctrl_snap;
    p.selector = (o->mode == GPOP_MODE_LEARNED) ? selector_device_params_transposed() : nullptr;
    p.list = rb->sc_list; p.list_count = &rb->ctrl->n_sc_units; p.counter_slot = 0; p.dry = 0; p.t_task = nullptr;
    p.t_gpc = nullptr;
    p.log_both = o->mode == GPOP_MODE_LOG_BOTH && o->log_buffer && o->log_capacity;
    if (p.log_both && !rb->shadow) {
        cudaError_t ae = cudaSuccess;
        auto A = [&](auto **ptr, uint64_t n) {
            if (ae == cudaSuccess) ae = dalloc(g, ptr, n);
        };
        A(&rb->shadow, g->npng_pad);
        A(&rb->all_list, sc_unit_capacity(g));
        A(&rb->part_va, g->k);
        A(&rb->part_ea, g->k);
        A(&rb->t_pc, g->nst);
        A(&rb->t_sc, g->k);
        A(&rb->t_gpc, 1);
        A(&rb->t_gsc, 1);
        A(&rb->feat, 8ull * g->k);
        if (ae != cudaSuccess) return fail(GPOP_ERR_OOM, std::string("LOG_BOTH buffers: ") + cudaGetErrorString(ae));
    }
    p.all_list = rb->all_list; p.feat = rb->feat; p.part_va = rb->part_va; p.part_ea = rb->part_ea;
    // a resumed run continues the saved state: iterations are numbered on from it (BFS levels), the cap
    // counts this call's iterations, and its first plan tests the saved L1 change
    const bool resume = o->resume != 0;
    if (resume && rb->state_algo != ALGO) return fail(GPOP_ERR_INVALID_ARG, "resume: no saved state of this algorithm");
    if (resume) {  // the options that shape the result must be those of the saved run
        const bool src = ALGO == ALG_BFS || ALGO == ALG_SSSP || ALGO == ALG_PPR || ALGO == ALG_NIBBLE;
        const bool damp = ALGO == ALG_PR || ALGO == ALG_PPR;
        if (src && o->source != rb->state_source)
            return fail(GPOP_ERR_INVALID_ARG, "resume: another source than the saved run's");
        if (damp && o->damping != rb->state_damping)
            return fail(GPOP_ERR_INVALID_ARG, "resume: another damping than the saved run's");
        if (ALGO == ALG_NIBBLE && o->epsilon != rb->state_epsilon)
            return fail(GPOP_ERR_INVALID_ARG, "resume: another threshold than the saved run's");
        if ((uint32_t)(B16 ? 1 : 0) != rb->state_bf16)
            return fail(GPOP_ERR_INVALID_ARG, "resume: another message format than the saved run's");
    }
    const uint32_t base = resume ? rb->state_iter : 0u;
    p.source = o->source; p.tol = o->tol_l1;
    p.max_iters = o->max_iters > 0xFFFFFFFEu - base ? 0xFFFFFFFEu : base + o->max_iters;
    p.t_res0 = resume ? rb->state_res : 0.0;
    rb->state_algo = -1;  // until this run succeeds
    if (ALGO == ALG_MSBFS) {
        p.msrc = mpass->src; p.nsrc = mpass->n; p.lvl_ms = mpass->lvl;
    }
    p.algo = ALGO; p.policy = o->mode == GPOP_MODE_LOG_BOTH ? GPOP_MODE_ANALYTIC : o->mode;
    p.bw_num = o->bw_ratio_num; p.bw_den = o->bw_ratio_den;
    p.isg_w = o->isg_waves >= 2 ? o->isg_waves : 0u;
    if (ALGO == ALG_PR) {
        p.c0 = (float)((1.0 - o->damping) / (double)g->V);
        p.c1 = (float)o->damping;
    } else if (ALGO == ALG_PPR) {
        p.c0 = (float)(1.0 - o->damping);
        p.c1 = (float)o->damping;
    } else if (ALGO == ALG_NIBBLE) {
        p.eps = (float)o->epsilon;
    }

    int grid_pc = 0, grid_sc = 0, grid_ga = 0;
    const size_t sc_smem = sizeof(uint32_t) * std::max<uint32_t>(g->max_row_subs, 1);
    GPOP_CUDA_TRY(cudaFuncSetAttribute(k_scatter_sc<ALGO, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sc_smem));
    // k_scatter_pc stages one partition's values (P words) in dynamic shared memory
    const size_t spc_smem = sizeof(uint32_t) * (size_t)g->P;
    GPOP_CUDA_TRY(cudaFuncSetAttribute(k_scatter_pc<B16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)spc_smem));
    grid_pc = persistent_grid(k_scatter_pc<B16>, kScatterPcThreads, spc_smem, g->num_sms);
    grid_sc = persistent_grid(k_scatter_sc<ALGO, B16>, kScatterThreads, sc_smem, g->num_sms);
    grid_ga = persistent_grid(k_gather<ALGO, B16>, kGatherThreads, 0, g->num_sms);
    // k_gather_pc: column accumulator and as many block value buffers as the opt-in shared memory holds
    // (at most kPcMaxBufs); dynamic shared memory is opted in explicitly
    size_t gpc_smem = 0;
    {
        cudaFuncAttributes fa;
        GPOP_CUDA_TRY(cudaFuncGetAttributes(&fa, k_gather_pc<ALGO, B16>));
        int optin = 0, dev = 0;
        GPOP_CUDA_TRY(cudaGetDevice(&dev));
        GPOP_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const size_t fixed = sizeof(uint32_t) * (size_t)g->P;
        const size_t buf = sizeof(uint32_t) * (kPcBlock + 4);
        const size_t avail = (size_t)optin > fixed + fa.sharedSizeBytes ? optin - fixed - fa.sharedSizeBytes : 0;
        const uint32_t nb = (uint32_t)std::min<size_t>(kPcMaxBufs, avail / buf);
        if (nb < 2) return fail(GPOP_ERR_INVALID_ARG, "partition size too large for the PC gather's shared memory");
        p.pc_nbuf = nb;
        gpc_smem = fixed + nb * buf;
        GPOP_CUDA_TRY(cudaFuncSetAttribute(k_gather_pc<ALGO, B16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)gpc_smem));
    }
    const int grid_gh = persistent_grid(k_gather_pc<ALGO, B16>, kPcThreads, gpc_smem, g->num_sms);

    // initial frontier (Alg. 4 driver: loadFrontier and initial values)
    p.epoch = ++g->epoch;
    // split-SC cursors are zero at rest; reset them in case an earlier run stopped part-way
    GPOP_CUDA_TRY(cudaMemsetAsync(rb->sc_gcur, 0, 4ull * std::max<uint64_t>(g->nsub, 1), s));
    GPOP_CUDA_TRY(cudaMemsetAsync(rb->sc_udone, 0, 4ull * g->k, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(rb->gath, 0, 8, s));
    rb->rate_pc = rb->rate_sc = 0.0;
    const bool learned = p.policy == GPOP_MODE_LEARNED && p.selector;
    p.col_done = learned ? rb->col_done : nullptr;
    if (learned) GPOP_CUDA_TRY(cudaMemsetAsync(rb->col_done, 0, 4ull * g->k, s));
    if (!resume) {
        if (ALGO == ALG_MSBFS) GPOP_CUDA_TRY(cudaMemsetAsync(p.lvl_ms, 0xFF, 4ull * p.nsrc * g->V, s));
        k_init<ALGO><<<std::max(1, std::min((int)((g->V / 32 + 255) / 256), 4096)), 256, 0, s>>>(p);
        if (ALGO == ALG_MSBFS) k_msbfs_sources<<<1, 32, 0, s>>>(p);
    } else {
        GPOP_CUDA_TRY(cudaMemsetAsync(&rb->ctrl->error, 0, 4, s));  // k_init's reset of the error word
    }
    k_task_stats<<<std::max(1, std::min((int)g->ngt, 8 * g->num_sms)), kGatherThreads, 0, s>>>(p);
    GPOP_CUDA_TRY(cudaGetLastError());

    cudaEvent_t ev0, ev1;
    GPOP_CUDA_TRY(cudaEventCreate(&ev0));
    GPOP_CUDA_TRY(cudaEventCreate(&ev1));
    gpop_run_stats st;
    memset(&st, 0, sizeof st);
    GPOP_CUDA_TRY(cudaEventRecord(ev0, s));
    // optional per-kernel CUDA-event timing: a start/stop pair per kernel kind, resolved at the
    // next host synchronisation (which the plan's control read provides every iteration)
    // Launches between two host synchronisations form a chain of events: one record before the first
    // launch and one after each, so that launch j takes from event j to event j + 1.
    // LOG_BOTH: events around the two shadow scatters of an iteration (their wall times)
    cudaEvent_t lev[3] = {};
    if (p.log_both)
        for (auto &ev : lev) GPOP_CUDA_TRY(cudaEventCreate(&ev));
    const bool prof = o->profile_kernels != 0;
    cudaEvent_t kev[8] = {};
    int kind_of[7] = {};
    int nchain = 0;  // launches in the chain
    if (prof)
        for (auto &ev : kev) GPOP_CUDA_TRY(cudaEventCreate(&ev));
    auto resolve = [&]() {
        for (int j = 0; j < nchain; ++j) {
            float kms = 0.f;
            cudaEventElapsedTime(&kms, kev[j], kev[j + 1]);
            st.kernel_ms[kind_of[j]] += kms;
            st.kernel_launches[kind_of[j]] += 1;
        }
        nchain = 0;
    };
    // launches an iteration kernel with programmatic stream serialisation (see GPOP_GRID_DEP); the first
    // failed launch is kept in launch_err
    cudaError_t launch_err = cudaSuccess;
    auto launch_dep = [&](auto kernel, uint32_t grid, uint32_t block, size_t smem, const Params &kp) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, kp);
        if (e != cudaSuccess && launch_err == cudaSuccess) launch_err = e;
    };
    auto timed = [&](int kind, auto launch) {
        if (prof && nchain == 0) cudaEventRecord(kev[0], s);
        launch();
        if (prof) {
            kind_of[nchain] = kind;
            cudaEventRecord(kev[++nchain], s);
        }
    };
    uint32_t iter = 0;
    gpop_status status = GPOP_OK;
    // plan of iteration it (0-based): learned policy's first choices from k_select, later ones from the
    // previous gather's tail (the last task of each column)
    auto launch_plan = [&](uint32_t it, const Params &pp) {
        const bool first_select = learned && it == 0;
        timed(0, [&] {
            if (first_select)
                launch_dep(k_select, std::min<uint32_t>((g->k + kSelectWarps - 1) / kSelectWarps, 8u * g->num_sms),
                           32 * kSelectWarps, 0, pp);
            launch_dep(k_plan, 1, kPlanThreads, 0, pp);
        });
        if (prof && first_select) st.kernel_launches[0] += 1;  // k_select
    };
    // scatter and gather of one iteration, as the plan c decided
    const int grid_seg = std::max(1, std::min((int)(((uint64_t)g->k * ((g->P + 1023) / 1024) + 7) / 8), 16 * g->num_sms));
    auto launch_work = [&](const Params &pp, const Control &c) -> cudaError_t {
        // per-segment active edges of the partitions the SC scatter (or the LOG_BOTH shadow) will visit
        if (p.log_both || c.n_sc > 0) timed(2, [&] { launch_dep(k_sc_segments, grid_seg, 256, 0, pp); });
        if (p.log_both) {
            // time both modes for every partition picked this iteration (shadow launches first:
            // the real SC scatter below rewrites the same bins with the same pairs)
            cudaMemsetAsync(rb->t_gpc, 0, 8, s);
            cudaMemsetAsync(rb->t_gsc, 0, 8, s);
            Params q1 = pp;
            q1.pdata = rb->shadow; q1.dry = 1; q1.counter_slot = 3; q1.t_task = rb->t_pc;
            cudaEventRecord(lev[0], s);
            k_scatter_pc<B16><<<grid_pc, kScatterPcThreads, spc_smem, s>>>(q1);
            cudaEventRecord(lev[1], s);
            Params q2 = pp;
            q2.dry = 1; q2.counter_slot = 4; q2.list = rb->all_list; q2.list_count = &rb->counters[7];
            q2.t_task = rb->t_sc;
            cudaMemsetAsync(rb->t_sc, 0, 8ull * g->k, s);  // split partitions add their units' CTA times
            k_scatter_sc<ALGO, B16><<<grid_sc, kScatterThreads, sc_smem, s>>>(q2);
            cudaEventRecord(lev[2], s);
        }
        Params ps = pp;
        ps.counter_slot = 1;
        Params pg = pp;
        pg.t_gsc = p.log_both ? rb->t_gsc : nullptr;
        Params pgc = pp;
        pgc.t_gpc = p.log_both ? rb->t_gpc : nullptr;
        pgc.pc_skip = c.n_pc < g->k;  // some partition is not PC: skip blocks whose sources all are not
        if (c.n_pc + c.n_null > 0)
            timed(1, [&] { launch_dep(k_scatter_pc<B16>, grid_pc, kScatterPcThreads, spc_smem, pp); });
        if (c.n_sc > 0) timed(2, [&] { launch_dep(k_scatter_sc<ALGO, B16>, grid_sc, kScatterThreads, sc_smem, ps); });
        if (c.n_pc > 0) {
            timed(4, [&] { launch_dep(k_gather_pc<ALGO, B16>, grid_gh, kPcThreads, gpc_smem, pgc); });
            if (g->nmerge)
                timed(5, [&] { launch_dep(k_merge_pc<ALGO>, std::min<uint32_t>(g->nmerge, 16u * g->num_sms), 256, 0, pp); });
        }
        timed(3, [&] { launch_dep(k_gather<ALGO, B16>, grid_ga, kGatherThreads, 0, pg); });
        const cudaError_t e = cudaGetLastError();
        return launch_err != cudaSuccess ? launch_err : e;
    };
    // the plan's verdict on iteration iter: false when the loop stops (termination or error)
    auto take = [&](const Control &c) -> bool {
        if (c.error) {
            status = fail(GPOP_ERR_TIMEOUT, "a bounded mbarrier wait ran out");
            return false;
        }
        st.residual = c.residual;
        if (c.done) {
            st.converged = (c.frontier_v == 0) || ((ALGO == ALG_PR || ALGO == ALG_PPR) && base + iter > 0 && c.residual < o->tol_l1);
            return false;
        }
        ++iter;
        st.edges_scattered += c.frontier_e;
        st.vertices_scattered += c.frontier_v;
        st.pc_partition_steps += c.n_pc;
        st.sc_partition_steps += c.n_sc;
        st.model_bytes += c.model_bytes;
        st.sc_vertices_scattered += c.sc_v;
        st.sc_edges_scattered += c.sc_e;
        return true;
    };
    // Each iteration: the plan, the host's read of its snapshot (mapped memory written by k_plan, no copy
    // in the stream), then the launches the plan asks for
    for (;;) {
        p.iter = base + iter + 1;
        p.epoch = ++g->epoch;
        launch_plan(iter, p);
        cudaError_t ce = launch_err != cudaSuccess ? launch_err : cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { status = fail(GPOP_ERR_CUDA, std::string("plan: ") + cudaGetErrorString(ce)); break; }
        if (prof) resolve();
        const Control c = rb->h_ctrl[(base + iter) & 1];  // this plan's slot: (p.iter - 1) & 1
        if (!take(c)) break;
        if (o->trace_frontier) {
            o->trace_frontier[2 * (iter - 1)] = c.frontier_v;
            o->trace_frontier[2 * (iter - 1) + 1] = c.frontier_e;
        }
        if (o->trace_modes) {
            ce = cudaMemcpyAsync(o->trace_modes + (uint64_t)(iter - 1) * g->k, rb->mode, g->k, cudaMemcpyDeviceToHost, s);
            if (ce != cudaSuccess) { status = fail(GPOP_ERR_CUDA, cudaGetErrorString(ce)); break; }
        }
        ce = launch_work(p, c);
        if (ce != cudaSuccess) { status = fail(GPOP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(ce)); break; }
        if (p.log_both) {
            const double occ[3] = {(double)grid_pc / g->num_sms, (double)grid_sc / g->num_sms,
                                   (double)grid_ga / g->num_sms};
            status = log_iteration(g, rb, o, s, iter, &st, occ, lev);
            if (status != GPOP_OK) break;
        }
    }
    cudaEventRecord(ev1, s);
    cudaEventSynchronize(ev1);
    if (prof) {
        resolve();
        for (auto &ev : kev) cudaEventDestroy(ev);
    }
    if (p.log_both)
        for (auto &ev : lev) cudaEventDestroy(ev);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (status != GPOP_OK) {
        g->pdata_dirty = true;
        return status;
    }
    st.iterations = iter;
    st.device_ms = ms;
    {
        unsigned long long gv = 0;
        GPOP_CUDA_TRY(cudaMemcpy(&gv, rb->gath, 8, cudaMemcpyDeviceToHost));
        st.gathered_vertices = gv;
    }
    if (ALGO != ALG_MSBFS) {
        rb->state_algo = ALGO;
        rb->state_iter = base + iter;
        rb->state_res = st.residual;
        rb->state_source = o->source;
        rb->state_damping = o->damping;
        rb->state_epsilon = o->epsilon;
        rb->state_bf16 = B16 ? 1u : 0u;
    }

    // outputs
    cudaMemcpyKind kind = out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const uint32_t *res_src = (ALGO == ALG_BFS) ? rb->lvl : rb->val;
    if (ALGO != ALG_MSBFS && out_values) GPOP_CUDA_TRY(cudaMemcpyAsync(out_values, res_src, 4ull * g->V, kind, s));
    if (ALGO == ALG_BFS && out_parent) GPOP_CUDA_TRY(cudaMemcpyAsync(out_parent, rb->val, 4ull * g->V, kind, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    if (stats) *stats = st;
    return GPOP_OK;
}

}  // namespace gpop

using namespace gpop;

extern "C" void gpop_run_opts_default(gpop_run_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->algo = GPOP_PAGERANK;
    o->damping = 0.85;
    o->max_iters = 1000;
    o->tol_l1 = 0.0;
    o->mode = GPOP_MODE_ANALYTIC;
    o->bw_ratio_num = 2;
    o->bw_ratio_den = 1;
    o->epsilon = 1e-9;
}

// PC data rows in the run's message format and all-NULL where not written, and the run buffers
static gpop_status prepare_run(Graph *g, int fmt, cudaStream_t s, RunBuffers **out) {
    if (fmt != g->pdata_fmt) {  // rows written in the other message format must not be read as this one
        g->pdata_dirty = true;
        g->pdata_fmt = fmt;
    }
    if (g->pdata_dirty) {
        // a failed run may have left PC data rows partially written: restore the all-NULL state
        GPOP_CUDA_TRY(cudaMemsetAsync(g->pdata, 0xFF, 4ull * std::max<uint64_t>(g->npng_pad, 1), s));
        GPOP_CUDA_TRY(cudaMemsetAsync(g->pc_state, 0, g->k, s));
        g->pdata_dirty = false;
    }
    RunBuffers *rb = static_cast<RunBuffers *>(g->run);
    if (!rb) {
        gpop_status st = alloc_runbufs(g, &rb);
        if (st != GPOP_OK) return st;
        g->run = rb;
    }
    *out = rb;
    return GPOP_OK;
}

static gpop_status check_common_opts(const gpop_run_opts *o) {
    if (o->mode < GPOP_MODE_ANALYTIC || o->mode > GPOP_MODE_LOG_BOTH) return fail(GPOP_ERR_INVALID_ARG, "unknown mode policy");
    if (o->bw_ratio_num == 0 || o->bw_ratio_den == 0) return fail(GPOP_ERR_INVALID_ARG, "bandwidth ratio must be positive");
    if (o->mode == GPOP_MODE_LEARNED && !selector_device_params())
        return fail(GPOP_ERR_NO_SELECTOR, "learned mode requested but no selector is installed");
    return GPOP_OK;
}

extern "C" gpop_status gpop_run(gpop_graph *h, const gpop_run_opts *o, void *out_values, uint32_t *out_parent,
                                int out_is_device, gpop_run_stats *stats) {
    set_error("");
    if (!h || !o) return fail(GPOP_ERR_INVALID_ARG, "NULL graph or options");
    Graph *g = &h->g;
    if (o->algo < GPOP_PAGERANK || o->algo > GPOP_NIBBLE) return fail(GPOP_ERR_INVALID_ARG, "unknown algorithm");
    if ((o->algo == GPOP_BFS || o->algo == GPOP_SSSP || o->algo == GPOP_PPR || o->algo == GPOP_NIBBLE) &&
        o->source >= g->V)
        return fail(GPOP_ERR_INVALID_ARG, "source out of range");
    if (o->algo == GPOP_SSSP && !g->weighted) return fail(GPOP_ERR_INVALID_ARG, "SSSP needs a weighted graph");
    gpop_status cs = check_common_opts(o);
    if (cs != GPOP_OK) return cs;
    if (o->msg_bf16 && o->algo != GPOP_PAGERANK && o->algo != GPOP_PPR)
        return fail(GPOP_ERR_INVALID_ARG, "BF16 messages are for PageRank and PPR (the other algorithms keep FP32 / exact messages)");
    if ((o->algo == GPOP_PAGERANK || o->algo == GPOP_PPR) && !(o->damping > 0.0 && o->damping < 1.0))
        return fail(GPOP_ERR_INVALID_ARG, "damping must be in (0, 1)");
    if (o->algo == GPOP_NIBBLE && !(o->epsilon >= 0.0 && std::isfinite(o->epsilon)))
        return fail(GPOP_ERR_INVALID_ARG, "Nibble threshold must be finite and >= 0");
    if (o->isg_waves >= 2 && o->algo != GPOP_CC && o->algo != GPOP_SSSP)
        return fail(GPOP_ERR_INVALID_ARG, "interleaved scatter-gather is for CC and SSSP (monotone minimum applications)");
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    const int fmt = o->msg_bf16 ? 1 : 0;
    RunBuffers *rb = nullptr;
    gpop_status ps = prepare_run(g, fmt, s, &rb);
    if (ps != GPOP_OK) return ps;
    switch (o->algo) {
    case GPOP_PAGERANK:
        return fmt ? run_algo<ALG_PR, true>(g, rb, o, s, out_values, out_parent, out_is_device, stats)
                   : run_algo<ALG_PR, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    case GPOP_BFS: return run_algo<ALG_BFS, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    case GPOP_CC: return run_algo<ALG_CC, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    case GPOP_SSSP: return run_algo<ALG_SSSP, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    case GPOP_NIBBLE: return run_algo<ALG_NIBBLE, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    default:
        return fmt ? run_algo<ALG_PPR, true>(g, rb, o, s, out_values, out_parent, out_is_device, stats)
                   : run_algo<ALG_PPR, false>(g, rb, o, s, out_values, out_parent, out_is_device, stats);
    }
}

extern "C" gpop_status gpop_run_msbfs(gpop_graph *h, const gpop_run_opts *o, const uint32_t *sources,
                                      uint32_t num_sources, uint32_t *out_levels, int out_is_device,
                                      gpop_run_stats *stats) {
    set_error("");
    if (!h || !o) return fail(GPOP_ERR_INVALID_ARG, "NULL graph or options");
    if (num_sources && (!sources || !out_levels)) return fail(GPOP_ERR_INVALID_ARG, "NULL sources or level buffer");
    Graph *g = &h->g;
    for (uint32_t j = 0; j < num_sources; ++j)
        if (sources[j] >= g->V) return fail(GPOP_ERR_INVALID_ARG, "source out of range");
    if (o->msg_bf16) return fail(GPOP_ERR_INVALID_ARG, "BF16 messages are for PageRank and PPR (BFS stays exact)");
    if (o->resume) return fail(GPOP_ERR_INVALID_ARG, "multi-source BFS does not resume");
    if (o->isg_waves >= 2) return fail(GPOP_ERR_INVALID_ARG, "interleaved scatter-gather is for CC and SSSP");
    gpop_status cs = check_common_opts(o);
    if (cs != GPOP_OK) return cs;
    gpop_run_stats total;
    memset(&total, 0, sizeof total);
    total.converged = 1;
    if (num_sources == 0) {
        if (stats) *stats = total;
        return GPOP_OK;
    }
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    RunBuffers *rb = nullptr;
    gpop_status ps = prepare_run(g, 0, s, &rb);
    if (ps != GPOP_OK) return ps;
    if (!rb->msrc) {
        cudaError_t e = dalloc(g, &rb->msrc, kMsBfsWidth);
        if (e != cudaSuccess) return fail(GPOP_ERR_OOM, std::string("source list: ") + cudaGetErrorString(e));
    }
    if (!out_is_device && !rb->lvl_ms) {  // host output: one pass's level rows are staged on the device
        cudaError_t e = dalloc(g, &rb->lvl_ms, (uint64_t)kMsBfsWidth * g->V);
        if (e != cudaSuccess) return fail(GPOP_ERR_OOM, std::string("level rows: ") + cudaGetErrorString(e));
    }
    for (uint32_t b = 0; b < num_sources; b += kMsBfsWidth) {
        const uint32_t n = std::min<uint32_t>(kMsBfsWidth, num_sources - b);
        uint32_t *rows = out_levels + (uint64_t)b * g->V;
        GPOP_CUDA_TRY(cudaMemcpyAsync(rb->msrc, sources + b, 4ull * n, cudaMemcpyHostToDevice, s));
        MsPass mp{rb->msrc, n, out_is_device ? rows : rb->lvl_ms};
        gpop_run_stats st;
        gpop_status r = run_algo<ALG_MSBFS, false>(g, rb, o, s, nullptr, nullptr, 1, &st, &mp);
        if (r != GPOP_OK) return r;
        if (!out_is_device) {
            GPOP_CUDA_TRY(cudaMemcpyAsync(rows, rb->lvl_ms, 4ull * n * g->V, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        }
        total.iterations += st.iterations;
        total.converged &= st.converged;
        total.edges_scattered += st.edges_scattered;
        total.vertices_scattered += st.vertices_scattered;
        total.pc_partition_steps += st.pc_partition_steps;
        total.sc_partition_steps += st.sc_partition_steps;
        total.model_bytes += st.model_bytes;
        total.device_ms += st.device_ms;
        total.sc_vertices_scattered += st.sc_vertices_scattered;
        total.sc_edges_scattered += st.sc_edges_scattered;
        total.gathered_vertices += st.gathered_vertices;
        total.log_records += st.log_records;
        for (int i = 0; i < 6; ++i) {
            total.kernel_ms[i] += st.kernel_ms[i];
            total.kernel_launches[i] += st.kernel_launches[i];
        }
    }
    if (stats) *stats = total;
    return GPOP_OK;
}

// Graphs built as one disjoint union: the BFS levels of graph b0 + j (j < n) are row j of the pass's
// multi-source BFS over that graph's own vertices (no edge leaves a graph); one thread per vertex of the
// pass's graphs, the graph found by binary search over their first vertices
__global__ void k_union_levels(const uint32_t *rows, uint32_t V, const uint32_t *goff, uint32_t b0, uint32_t n,
                               uint32_t *out) {
    const uint32_t v0 = goff[b0], v1 = goff[b0 + n];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < v1 - v0; x += stride) {
        const uint32_t v = v0 + (uint32_t)x;
        uint32_t lo = 0, hi = n;  // the last j with goff[b0 + j] <= v
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (goff[b0 + mid] <= v) lo = mid; else hi = mid;
        }
        out[v] = rows[(uint64_t)lo * V + v];
    }
}

extern "C" gpop_status gpop_run_bfs_union(gpop_graph *h, const gpop_run_opts *o, const uint32_t *sources,
                                          uint32_t *out_levels, int out_is_device, gpop_run_stats *stats) {
    set_error("");
    if (!h || !o || !sources || !out_levels) return fail(GPOP_ERR_INVALID_ARG, "NULL argument");
    Graph *g = &h->g;
    if (g->goff.size() < 2) return fail(GPOP_ERR_INVALID_ARG, "the graph was not built by gpop_graph_build_union");
    const uint32_t ng = (uint32_t)g->goff.size() - 1;
    for (uint32_t i = 0; i < ng; ++i)
        if (sources[i] >= g->goff[i + 1] - g->goff[i]) return fail(GPOP_ERR_INVALID_ARG, "source out of its graph's range");
    if (o->msg_bf16 || o->resume || o->isg_waves >= 2)
        return fail(GPOP_ERR_INVALID_ARG, "msg_bf16, resume and isg_waves must be 0");
    gpop_status cs = check_common_opts(o);
    if (cs != GPOP_OK) return cs;
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    RunBuffers *rb = nullptr;
    gpop_status ps = prepare_run(g, 0, s, &rb);
    if (ps != GPOP_OK) return ps;
    if (!rb->msrc) {
        cudaError_t e = dalloc(g, &rb->msrc, kMsBfsWidth);
        if (e != cudaSuccess) return fail(GPOP_ERR_OOM, std::string("source list: ") + cudaGetErrorString(e));
    }
    if (!rb->lvl_ms) {  // one pass's level rows (32 x V)
        cudaError_t e = dalloc(g, &rb->lvl_ms, (uint64_t)kMsBfsWidth * g->V);
        if (e != cudaSuccess) return fail(GPOP_ERR_OOM, std::string("level rows: ") + cudaGetErrorString(e));
    }
    uint32_t *d_goff = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc(&d_goff, 4ull * (ng + 1));
    if (e == cudaSuccess && !out_is_device) e = cudaMalloc(&d_out, 4ull * g->V);
    if (e != cudaSuccess) {
        cudaFree(d_goff);
        return fail(GPOP_ERR_OOM, std::string("union buffers: ") + cudaGetErrorString(e));
    }
    gpop_run_stats total;
    memset(&total, 0, sizeof total);
    total.converged = 1;
    gpop_status status = GPOP_OK;
    e = cudaMemcpyAsync(d_goff, g->goff.data(), 4ull * (ng + 1), cudaMemcpyHostToDevice, s);
    uint32_t *dst = out_is_device ? out_levels : d_out;
    std::vector<uint32_t> src(kMsBfsWidth);
    for (uint32_t b0 = 0; b0 < ng && e == cudaSuccess; b0 += kMsBfsWidth) {
        const uint32_t n = std::min<uint32_t>(kMsBfsWidth, ng - b0);
        for (uint32_t j = 0; j < n; ++j) src[j] = g->goff[b0 + j] + sources[b0 + j];
        e = cudaMemcpyAsync(rb->msrc, src.data(), 4ull * n, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        MsPass mp{rb->msrc, n, rb->lvl_ms};
        gpop_run_stats st;
        status = run_algo<ALG_MSBFS, false>(g, rb, o, s, nullptr, nullptr, 1, &st, &mp);
        if (status != GPOP_OK) break;
        const uint32_t nv = g->goff[b0 + n] - g->goff[b0];
        k_union_levels<<<std::max(1u, std::min((nv + 255) / 256, 8u * g->num_sms)), 256, 0, s>>>(rb->lvl_ms, g->V, d_goff,
                                                                                               b0, n, dst);
        e = cudaGetLastError();
        total.iterations += st.iterations;
        total.converged &= st.converged;
        total.edges_scattered += st.edges_scattered;
        total.vertices_scattered += st.vertices_scattered;
        total.pc_partition_steps += st.pc_partition_steps;
        total.sc_partition_steps += st.sc_partition_steps;
        total.model_bytes += st.model_bytes;
        total.device_ms += st.device_ms;
        total.sc_vertices_scattered += st.sc_vertices_scattered;
        total.sc_edges_scattered += st.sc_edges_scattered;
        total.gathered_vertices += st.gathered_vertices;
        for (int i = 0; i < 6; ++i) {
            total.kernel_ms[i] += st.kernel_ms[i];
            total.kernel_launches[i] += st.kernel_launches[i];
        }
    }
    if (status == GPOP_OK && e == cudaSuccess && !out_is_device)
        e = cudaMemcpyAsync(out_levels, d_out, 4ull * g->V, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_goff);
    if (d_out) cudaFree(d_out);
    if (status != GPOP_OK) return status;
    if (e != cudaSuccess) return fail(GPOP_ERR_CUDA, std::string("union BFS: ") + cudaGetErrorString(e));
    if (stats) *stats = total;
    return GPOP_OK;
}

extern "C" gpop_status gpop_probe_bounded_wait(uint32_t tries, uint32_t *gave_up) {
    set_error("");
    if (!gave_up) return fail(GPOP_ERR_INVALID_ARG, "gave_up is NULL");
    if (tries > kPcSpinLimit) return fail(GPOP_ERR_INVALID_ARG, "tries above the engine's own limit (2^24)");
    uint32_t *d_err = nullptr;
    GPOP_CUDA_TRY(cudaMalloc((void **)&d_err, 4));
    uint32_t h = 0;
    cudaError_t e = cudaMemset(d_err, 0, 4);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(tries, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_err, 4, cudaMemcpyDeviceToHost);
    cudaFree(d_err);
    if (e != cudaSuccess) return fail(GPOP_ERR_CUDA, std::string("wait probe: ") + cudaGetErrorString(e));
    if (h & 2u) return fail(GPOP_ERR_DEVICE_CHECK, "a barrier phase that nothing completes reported completion");
    *gave_up = h & 1u;
    return GPOP_OK;
}

// --- checkpoint ---------------------------------------------------------------------------------

namespace {
// version 2: the graph (vertex and edge counts, partition size, fingerprint of its edges and weights) and
// the options of the saved run that shape its result, so that a checkpoint is never continued on another
// graph or with other options
struct StateHeader {
    uint32_t magic, version;
    int32_t algo;
    uint32_t V, iterations, nwords;
    double residual;
    uint64_t E, fingerprint;
    uint32_t P, msg_bf16, source, pad;
    double damping, epsilon;
};
static_assert(sizeof(StateHeader) == 80, "checkpoint header is 80 bytes");
constexpr uint32_t kStateVersion = 2;
constexpr uint32_t kStateMagic = 0x54535047u;  // "GPST"
uint64_t state_bytes(uint32_t V) { return sizeof(StateHeader) + 12ull * V + 4ull * ((V + 31) / 32); }
}  // namespace

extern "C" gpop_status gpop_state_export(const gpop_graph *h, void *buffer, uint64_t capacity, uint64_t *size) {
    set_error("");
    if (!h || !size) return fail(GPOP_ERR_INVALID_ARG, "NULL graph or size");
    const Graph *g = &h->g;
    const RunBuffers *rb = static_cast<const RunBuffers *>(g->run);
    if (!rb || rb->state_algo < 0) return fail(GPOP_ERR_INVALID_ARG, "no run state to export");
    const uint64_t need = state_bytes(g->V);
    *size = need;
    if (!buffer) return GPOP_OK;
    if (capacity < need) return fail(GPOP_ERR_INVALID_ARG, "checkpoint buffer too small");
    StateHeader hd{};
    hd.magic = kStateMagic;
    hd.version = kStateVersion;
    hd.algo = rb->state_algo;
    hd.V = g->V;
    hd.iterations = rb->state_iter;
    hd.nwords = (g->V + 31) / 32;
    hd.residual = rb->state_res;
    hd.E = g->E;
    hd.fingerprint = g->fingerprint;
    hd.P = g->P;
    hd.msg_bf16 = rb->state_bf16;
    hd.source = rb->state_source;
    hd.damping = rb->state_damping;
    hd.epsilon = rb->state_epsilon;
    char *out = static_cast<char *>(buffer);
    memcpy(out, &hd, sizeof hd);
    out += sizeof hd;
    GPOP_CUDA_TRY(cudaDeviceSynchronize());
    GPOP_CUDA_TRY(cudaMemcpy(out, rb->val, 4ull * g->V, cudaMemcpyDeviceToHost));
    GPOP_CUDA_TRY(cudaMemcpy(out + 4ull * g->V, rb->lvl, 4ull * g->V, cudaMemcpyDeviceToHost));
    GPOP_CUDA_TRY(cudaMemcpy(out + 8ull * g->V, rb->sval, 4ull * g->V, cudaMemcpyDeviceToHost));
    GPOP_CUDA_TRY(cudaMemcpy(out + 12ull * g->V, rb->bits, 4ull * hd.nwords, cudaMemcpyDeviceToHost));
    return GPOP_OK;
}

extern "C" gpop_status gpop_state_import(gpop_graph *h, const void *buffer, uint64_t size) {
    set_error("");
    if (!h || !buffer) return fail(GPOP_ERR_INVALID_ARG, "NULL graph or buffer");
    Graph *g = &h->g;
    if (size < sizeof(StateHeader)) return fail(GPOP_ERR_INVALID_ARG, "checkpoint shorter than its header");
    StateHeader hd;
    memcpy(&hd, buffer, sizeof hd);
    if (hd.magic != kStateMagic || hd.version != kStateVersion)
        return fail(GPOP_ERR_INVALID_ARG, "not a checkpoint of this format");
    if (hd.V != g->V || size != state_bytes(g->V) || hd.nwords != (g->V + 31) / 32)
        return fail(GPOP_ERR_INVALID_ARG, "checkpoint of a graph with another vertex count");
    if (hd.E != g->E || hd.fingerprint != g->fingerprint)
        return fail(GPOP_ERR_INVALID_ARG, "checkpoint of another graph (its edges or weights differ)");
    if (hd.P != g->P) return fail(GPOP_ERR_INVALID_ARG, "checkpoint of another partition size");
    if (hd.msg_bf16 > 1) return fail(GPOP_ERR_INVALID_ARG, "checkpoint with an unknown message format");
    if (hd.algo < GPOP_PAGERANK || hd.algo > GPOP_NIBBLE) return fail(GPOP_ERR_INVALID_ARG, "checkpoint of an unknown algorithm");
    RunBuffers *rb = static_cast<RunBuffers *>(g->run);
    if (!rb) {
        gpop_status st = alloc_runbufs(g, &rb);
        if (st != GPOP_OK) return st;
        g->run = rb;
    }
    const char *in = static_cast<const char *>(buffer) + sizeof hd;
    GPOP_CUDA_TRY(cudaDeviceSynchronize());
    GPOP_CUDA_TRY(cudaMemcpy(rb->val, in, 4ull * g->V, cudaMemcpyHostToDevice));
    GPOP_CUDA_TRY(cudaMemcpy(rb->lvl, in + 4ull * g->V, 4ull * g->V, cudaMemcpyHostToDevice));
    GPOP_CUDA_TRY(cudaMemcpy(rb->sval, in + 8ull * g->V, 4ull * g->V, cudaMemcpyHostToDevice));
    GPOP_CUDA_TRY(cudaMemcpy(rb->bits, in + 12ull * g->V, 4ull * hd.nwords, cudaMemcpyHostToDevice));
    rb->state_algo = hd.algo;
    rb->state_iter = hd.iterations;
    rb->state_res = hd.residual;
    rb->state_source = hd.source;
    rb->state_damping = hd.damping;
    rb->state_epsilon = hd.epsilon;
    rb->state_bf16 = hd.msg_bf16;
    return GPOP_OK;
}
