// Batched seeded personalized PageRank (gpop_run_ppr_batch): up to 32 seeds per pass through the
// partition-centric scatter / gather of Alg. 2 on the PC layout of Alg. 3, every message carrying one FP32
// value per seed (lane j of a warp holds seed j).
//
// One pass = per iteration:
//   k_bscatter  every partition holding an active vertex (for any seed: the union frontier) writes, for
//               each slot of its PNG row, the 32 message values x_j[u] / deg(u) of the slot's source u;
//   k_bgather   one CTA per PC gather task (a range of one column's blocks): each block's PNG slots are
//               mapped in shared memory, and each warp folds the entries of its destination slice (the
//               same slice in every block of the task) into the column accumulator acc[P][32], lane j
//               adding seed j's values: 128-byte loads, no bank conflicts, no atomics, a fixed order;
//   k_bmerge    the partial vectors of columns split over several tasks, summed in task order;
//   k_bfilter   x_j = alpha [v = s_j] + (1 - alpha) acc_j for every vertex, the next messages, the union
//               frontier and each seed's L1 change (FP32 per 32 vertices, FP64 across them).
// Every partition with an active vertex is scattered in PC mode: a (destination, 32-value) pair would
// cost 132 bytes per active edge, against 128 bytes per PNG slot; and since a PPR vector's support only
// grows, a row written once stays current (rows start at zero: the sum's identity).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gpop_internal.cuh"

namespace gpop {
namespace {

constexpr uint32_t kSeeds = 32;                  // seeds per pass, one lane each
constexpr uint32_t kBatchMaxP = 1024;            // acc[P][32] floats must fit in shared memory
constexpr int kBThreads = 256;                   // scatter / filter CTAs
constexpr int kBGWarps = kPcGatherWarps;         // gather warps: one destination slice of each task each
constexpr int kBGThreads = 32 * kBGWarps;

struct BParams {
    uint32_t V, P, shift, k, npct, nmerge;
    const uint32_t *rowptr, *Ep;
    const uint16_t *png;
    const uint32_t *row_png, *row_bin, *bin_q;
    const uint4 *pc_runs, *pc_task;
    const uint32_t *pc_tsp, *pc_wsp, *pc_blk_run, *pe, *col_ntask, *col_part0;
    const uint2 *pc_merge;
    const uint32_t *seed;     // [32]: the pass's seeds, kNull for unused lanes
    float *X, *M, *S;         // V x 32 each: values, next messages, combined messages of the iteration
    float *pdata, *part;      // PNG slots x 32; partial vectors of split columns (npart x P x 32)
    uint32_t *bits;           // union frontier
    uint8_t *pact, *pact_prev, *pact_next;  // partitions with an active vertex: now, last iteration, next
    uint32_t *gflag;          // column received messages this iteration (== epoch)
    uint32_t *counter;        // gather task counter
    unsigned long long *edges;  // out-edges of the scattered partitions, summed over iterations
    double *res_part;         // per filter CTA and seed: L1 change
    double *res;              // per seed: L1 change of the iteration
    float c0, c1;             // alpha, 1 - alpha
    uint32_t epoch;
};

// seeds: value 1 and message 1 / deg on their own lane (FP32, as the single-seed run computes it)
__global__ void k_binit(BParams p) {
    const uint32_t j = threadIdx.x;
    if (j >= kSeeds) return;
    const uint32_t s = p.seed[j];
    if (s == kNull) return;
    const uint32_t deg = p.rowptr[s + 1] - p.rowptr[s];
    p.X[(uint64_t)s * kSeeds + j] = 1.f;
    p.M[(uint64_t)s * kSeeds + j] = deg ? 1.f / (float)deg : 0.f;
    atomicOr(&p.bits[s >> 5], 1u << (s & 31));
    p.pact[s >> p.shift] = 1;
}

// PC scatter (Alg. 3) of every partition with an active vertex; a partition that was active last
// iteration and no longer is has its row cleared (the sum's identity)
__global__ void __launch_bounds__(kBThreads) k_bscatter(BParams p) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kBThreads / 32;
    for (uint32_t q = blockIdx.x; q < p.k; q += gridDim.x) {
        const bool act = p.pact[q] != 0;
        if (!act && !p.pact_prev[q]) continue;
        if (act) {
            for (uint32_t b = p.row_bin[q] + threadIdx.x; b < p.row_bin[q + 1]; b += kBThreads)
                p.gflag[p.bin_q[b]] = p.epoch;
            if (threadIdx.x == 0) atomicAdd(p.edges, (unsigned long long)p.Ep[q]);
        }
        const uint64_t g0 = (uint64_t)q << p.shift;
        // 32 slots per warp round: lane i reads slot i's source; then each quarter-warp copies one slot's
        // 128 bytes as eight 16-byte words, four slots at a time, eight loads in flight per lane
        const uint32_t r0 = p.row_png[q], r1 = p.row_png[q + 1];
        const uint32_t sub = (uint32_t)lane >> 3, l8 = (uint32_t)lane & 7u;
        uint32_t u_next = 0;
        if (r0 + (uint32_t)wid * 32 < r1)
            u_next = (uint32_t)lane < r1 - (r0 + (uint32_t)wid * 32) ? p.png[r0 + (uint32_t)wid * 32 + lane] : 0u;
        for (uint32_t base = r0 + (uint32_t)wid * 32; base < r1; base += (uint32_t)nw * 32) {
            const uint32_t n = min(32u, r1 - base);
            const uint32_t u_lane = u_next;  // this round's sources; the next round's load while copying
            const uint32_t nb = base + (uint32_t)nw * 32;
            if (nb < r1) u_next = (uint32_t)lane < r1 - nb ? p.png[nb + lane] : 0u;
            float4 v[8];
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                const uint32_t sl = k * 4 + sub;
                const uint32_t u = __shfl_sync(0xffffffffu, u_lane, (int)sl);
                v[k] = (act && sl < n) ? reinterpret_cast<const float4 *>(p.M + (g0 + u) * kSeeds)[l8]
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                const uint32_t sl = k * 4 + sub;
                if (sl < n) reinterpret_cast<float4 *>(p.pdata + (uint64_t)(base + sl) * kSeeds)[l8] = v[k];
            }
        }
    }
}

// PC gather: one CTA per task (1 per SM, persistent), acc[P][32] and the block's slot map in shared memory
__global__ void __launch_bounds__(kBGThreads, 1) k_bgather(BParams p) {
    extern __shared__ __align__(16) float s_acc[];                   // P x 32 (destination positions swizzled)
    uint32_t *s_map = reinterpret_cast<uint32_t *>(s_acc + (size_t)p.P * kSeeds);  // kPcBlock PNG slots
    __shared__ uint32_t s_task;
    constexpr uint32_t kSp = kPcGatherWarps + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(p.counter, 1u);
        __syncthreads();
        const uint32_t t = s_task;
        __syncthreads();
        if (t >= p.npct) break;
        const uint4 tk = p.pc_task[t];  // column, first block, end block, partial slot
        if (p.gflag[tk.x] != p.epoch) continue;
        for (uint32_t i = threadIdx.x; i < p.P * kSeeds; i += kBGThreads) s_acc[i] = 0.f;
        const uint32_t tsp = p.pc_tsp[t];
        for (uint32_t b = tk.y; b < tk.z; ++b) {
            __syncthreads();  // the accumulator is cleared and the previous block's map is no longer read
            // PNG slot of each staged message of the block, from its bin runs
            for (uint32_t r = p.pc_blk_run[b] + wid; r < p.pc_blk_run[b + 1]; r += kBGWarps) {
                const uint4 run = p.pc_runs[r];  // row-major source slot, length, offset in the block
                for (uint32_t o = lane; o < run.y; o += 32) s_map[run.z + o] = run.x + o;
            }
            __syncthreads();
            const uint32_t *sp = p.pc_wsp + (uint64_t)(tsp + (b - tk.y)) * kSp;
            const uint32_t e0 = sp[wid], e1 = sp[wid + 1];
            // the warp's entries (their order is immaterial: the warp alone owns these destinations; lane j
            // adds seed j's value of each entry in the order of the layout, a fixed order)
            uint32_t ent_next = (uint32_t)lane < e1 - min(e0, e1) ? p.pe[e0 + lane] : kPcPadIdx;
            for (uint32_t base = e0; base < e1; base += 32) {
                const uint32_t n = min(32u, e1 - base);
                const uint32_t ent = ent_next;
                if (base + 32 < e1)  // the next group's entries, loading while this group is folded
                    ent_next = (uint32_t)lane < e1 - base - 32 ? p.pe[base + 32 + lane] : kPcPadIdx;
                // lane i resolves entry i: its accumulator word and the PNG slot of its value
                const uint32_t idx = ent & 0xFFFFu;
                const bool real = (uint32_t)lane < n && idx < kPcBlock;  // padding entries fold nothing
                const uint32_t a_l = real ? (ent >> 16) * kSeeds : 0xFFFFFFFFu;
                const uint32_t slot_l = s_map[real ? idx : 0u];
#pragma unroll 1
                for (uint32_t k0 = 0; k0 < n; k0 += 16) {
                    float v[16];
                    uint32_t a[16];
#pragma unroll
                    for (uint32_t k = 0; k < 16; ++k) {
                        a[k] = __shfl_sync(0xffffffffu, a_l, (int)((k0 + k) & 31));
                        const uint32_t slot = __shfl_sync(0xffffffffu, slot_l, (int)((k0 + k) & 31));
                        if (k0 + k >= n) a[k] = 0xFFFFFFFFu;
                        v[k] = a[k] != 0xFFFFFFFFu ? p.pdata[(uint64_t)slot * kSeeds + lane] : 0.f;
                    }
#pragma unroll
                    for (uint32_t k = 0; k < 16; ++k)
                        if (a[k] != 0xFFFFFFFFu) s_acc[a[k] + lane] += v[k];
                }
            }
        }
        __syncthreads();
        const uint32_t gq = tk.x << p.shift, wq = min(p.P, p.V - gq);
        float *out = tk.w == kNull ? p.S + (uint64_t)gq * kSeeds : p.part + (uint64_t)tk.w * p.P * kSeeds;
        for (uint32_t i = threadIdx.x; i < wq * kSeeds; i += kBGThreads)
            out[i] = s_acc[pc_swz(i / kSeeds) * kSeeds + (i % kSeeds)];
        __syncthreads();
    }
}

// columns split over several gather tasks: their partial vectors summed in task order, per chunk of
// 1024 destinations
__global__ void __launch_bounds__(kBThreads) k_bmerge(BParams p) {
    for (uint32_t it = blockIdx.x; it < p.nmerge; it += gridDim.x) {
        const uint2 m = p.pc_merge[it];  // column, first destination
        if (p.gflag[m.x] != p.epoch) continue;
        const uint32_t gq = m.x << p.shift, wq = min(p.P, p.V - gq);
        const uint32_t nt = p.col_ntask[m.x], part0 = p.col_part0[m.x];
        const uint32_t d1 = min(wq, m.y + 1024);
        for (uint32_t i = m.y * kSeeds + threadIdx.x; i < d1 * kSeeds; i += kBThreads) {
            float s = 0.f;
            for (uint32_t t = 0; t < nt; ++t) s += p.part[((uint64_t)(part0 + t) * p.P) * kSeeds + i];
            p.S[(uint64_t)gq * kSeeds + i] = s;
        }
    }
}

// filter (PPR's filterFunc for every seed): x_j = alpha [v = s_j] + (1 - alpha) acc_j, message x_j / deg,
// the union frontier (a vertex is active when any seed's value is positive) and the L1 change per seed;
// one warp per 32-vertex frontier word, lane j = seed j
__global__ void __launch_bounds__(kBThreads) k_bfilter(BParams p) {
    __shared__ double s_res[kBThreads / 32][kSeeds];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nwords = (p.V + 31) / 32;
    const uint32_t seed = p.seed[lane];
    double dres = 0.0;
    for (uint32_t w = blockIdx.x * (kBThreads / 32) + wid; w < nwords; w += gridDim.x * (kBThreads / 32)) {
        const uint32_t v0 = w * 32, q = v0 >> p.shift;
        const bool got = p.gflag[q] == p.epoch && p.col_ntask[q] > 0;  // the column's messages were combined
        const uint32_t nv = min(32u, p.V - v0);
        const uint32_t rp_lane = p.rowptr[v0 + min((uint32_t)lane, nv)];  // row offsets, one per lane
        const uint32_t rp_last = p.rowptr[v0 + nv];
        uint32_t word = 0;
        float res = 0.f;
        for (uint32_t k0 = 0; k0 < nv; k0 += 8) {  // eight vertices at a time, their loads first
            float acc[8], xo[8];
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                const uint64_t o = (uint64_t)(v0 + k0 + k) * kSeeds + lane;
                const bool in = k0 + k < nv;
                acc[k] = (in && got) ? p.S[o] : 0.f;
                xo[k] = in ? p.X[o] : 0.f;
            }
#pragma unroll
            for (uint32_t k = 0; k < 8; ++k) {
                const uint32_t kk = k0 + k, v = v0 + kk;
                const uint32_t r0 = __shfl_sync(0xffffffffu, rp_lane, (int)(kk & 31));
                const uint32_t r1 = kk + 1 < nv ? __shfl_sync(0xffffffffu, rp_lane, (int)((kk + 1) & 31)) : rp_last;
                if (kk >= nv) continue;
                const uint64_t o = (uint64_t)v * kSeeds + lane;
                const float xn = fmaf(p.c1, acc[k], v == seed ? p.c0 : 0.f);
                const uint32_t deg = r1 - r0;
                p.X[o] = xn;
                p.M[o] = deg ? xn / (float)deg : 0.f;
                res += fabsf(xn - xo[k]);
                if (__any_sync(0xffffffffu, xn > 0.f)) word |= 1u << kk;
            }
        }
        if (lane == 0) {
            p.bits[w] = word;
            if (word) p.pact_next[q] = 1;
        }
        dres += (double)res;
    }
    s_res[wid][lane] = dres;
    __syncthreads();
    if (wid == 0) {
        double r = 0.0;
        for (int i = 0; i < kBThreads / 32; ++i) r += s_res[i][lane];
        p.res_part[(uint64_t)blockIdx.x * kSeeds + lane] = r;
    }
}

// each seed's L1 change: the filter CTAs' partials summed in CTA order
__global__ void k_bres(BParams p, uint32_t nparts) {
    const uint32_t j = threadIdx.x;
    if (j >= kSeeds) return;
    double r = 0.0;
    for (uint32_t b = 0; b < nparts; ++b) r += p.res_part[(uint64_t)b * kSeeds + j];
    p.res[j] = r;
}

// rows of the result: out[j][v] = X[v][j] for the pass's seeds, through 32 x 32 shared tiles
__global__ void k_btranspose(const float *X, float *out, uint32_t V, uint32_t nseeds) {
    __shared__ float tile[32][33];
    const uint32_t v0 = blockIdx.x * 32;
    for (uint32_t r = threadIdx.y; r < 32; r += blockDim.y) {
        const uint32_t v = v0 + r;
        tile[r][threadIdx.x] = v < V ? X[(uint64_t)v * kSeeds + threadIdx.x] : 0.f;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.y; j < nseeds; j += blockDim.y) {
        const uint32_t v = v0 + threadIdx.x;
        if (v < V) out[(uint64_t)j * V + v] = tile[threadIdx.x][j];
    }
}

struct BatchBuffers {
    std::vector<void *> ptrs;
    ~BatchBuffers() {
        for (void *q : ptrs) cudaFree(q);
    }
    template <typename T>
    cudaError_t alloc(T **q, uint64_t n) {
        void *r = nullptr;
        cudaError_t e = cudaMalloc(&r, std::max<uint64_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(r);
        *q = static_cast<T *>(r);
        return e;
    }
};

}  // namespace
}  // namespace gpop

using namespace gpop;

extern "C" gpop_status gpop_run_ppr_batch(gpop_graph *h, const gpop_run_opts *o, const uint32_t *seeds,
                                          uint32_t num_seeds, float *out_values, int out_is_device,
                                          gpop_run_stats *stats) {
    set_error("");
    if (!h || !o) return fail(GPOP_ERR_INVALID_ARG, "NULL graph or options");
    Graph *g = &h->g;
    if (num_seeds && (!seeds || !out_values)) return fail(GPOP_ERR_INVALID_ARG, "NULL seeds or output buffer");
    for (uint32_t j = 0; j < num_seeds; ++j)
        if (seeds[j] >= g->V) return fail(GPOP_ERR_INVALID_ARG, "seed out of range");
    if (!(o->damping > 0.0 && o->damping < 1.0)) return fail(GPOP_ERR_INVALID_ARG, "damping must be in (0, 1)");
    if (o->msg_bf16 || o->resume) return fail(GPOP_ERR_INVALID_ARG, "batched PPR: msg_bf16 and resume must be 0");
    if (g->P > kBatchMaxP)
        return fail(GPOP_ERR_INVALID_ARG, "batched PPR keeps 32 values per destination in shared memory: partition "
                                          "size must be at most 1024");
    gpop_run_stats total;
    memset(&total, 0, sizeof total);
    total.converged = 1;
    if (num_seeds == 0) {
        if (stats) *stats = total;
        return GPOP_OK;
    }
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    const size_t gsmem = sizeof(float) * (size_t)g->P * kSeeds + sizeof(uint32_t) * kPcBlock;
    {
        int optin = 0, dev = 0;
        GPOP_CUDA_TRY(cudaGetDevice(&dev));
        GPOP_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (gsmem + 64 > (size_t)optin) return fail(GPOP_ERR_INVALID_ARG, "batched PPR: shared memory too small");
        GPOP_CUDA_TRY(cudaFuncSetAttribute(k_bgather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem));
    }
    BatchBuffers bb;
    BParams p{};
    p.V = g->V; p.P = g->P; p.shift = g->shift; p.k = g->k; p.npct = g->npct; p.nmerge = g->nmerge;
    p.rowptr = g->rowptr; p.Ep = g->Ep; p.png = g->png; p.row_png = g->row_png; p.row_bin = g->row_bin;
    p.bin_q = g->bin_q; p.pc_runs = g->pc_runs; p.pc_task = g->pc_task; p.pc_tsp = g->pc_tsp; p.pc_wsp = g->pc_wsp;
    p.pc_blk_run = g->pc_blk_run; p.pe = g->pe; p.col_ntask = g->col_ntask; p.col_part0 = g->col_part0;
    p.pc_merge = g->pc_merge;
    p.c0 = (float)(1.0 - o->damping);
    p.c1 = (float)o->damping;
    const uint64_t V32 = (uint64_t)g->V * kSeeds, nw = (g->V + 31) / 32;
    const int grid_f = std::max(1, std::min((int)((nw + 7) / 8), 8 * g->num_sms));
    uint32_t *d_seed = nullptr;
    uint8_t *pa[3] = {};
    float *staging = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto **ptr, uint64_t n) {
        if (e == cudaSuccess) e = bb.alloc(ptr, n);
    };
    A(&p.X, V32); A(&p.M, V32); A(&p.S, V32);
    A(&p.pdata, g->npng_pad * kSeeds);
    A(&p.part, (uint64_t)g->npart * g->P * kSeeds);
    A(&p.bits, nw + 1);
    A(&pa[0], g->k); A(&pa[1], g->k); A(&pa[2], g->k);
    A(&p.gflag, g->k);
    A(&p.counter, 1);
    A(&p.edges, 1);
    A(&p.res_part, (uint64_t)grid_f * kSeeds);
    A(&p.res, kSeeds);
    A(&d_seed, kSeeds);
    if (!out_is_device) A(&staging, V32);
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? GPOP_ERR_OOM : GPOP_ERR_CUDA,
                    std::string("batched PPR buffers: ") + cudaGetErrorString(e));
    p.seed = d_seed;
    const bool prof = o->profile_kernels != 0;
    cudaEvent_t ev0, ev1, kev[2];
    GPOP_CUDA_TRY(cudaEventCreate(&ev0));
    GPOP_CUDA_TRY(cudaEventCreate(&ev1));
    GPOP_CUDA_TRY(cudaEventCreate(&kev[0]));
    GPOP_CUDA_TRY(cudaEventCreate(&kev[1]));
    auto timed = [&](int kind, auto launch) {
        if (prof) cudaEventRecord(kev[0], s);
        launch();
        if (prof) {
            cudaEventRecord(kev[1], s);
            cudaEventSynchronize(kev[1]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, kev[0], kev[1]);
            total.kernel_ms[kind] += ms;
            total.kernel_launches[kind] += 1;
        }
    };
    gpop_status status = GPOP_OK;
    uint32_t epoch = 0;
    GPOP_CUDA_TRY(cudaMemsetAsync(p.gflag, 0, 4ull * g->k, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(p.edges, 0, 8, s));
    GPOP_CUDA_TRY(cudaEventRecord(ev0, s));
    for (uint32_t b0 = 0; b0 < num_seeds && status == GPOP_OK; b0 += kSeeds) {
        const uint32_t n = std::min(kSeeds, num_seeds - b0);
        uint32_t hs[kSeeds];
        for (uint32_t j = 0; j < kSeeds; ++j) hs[j] = j < n ? seeds[b0 + j] : kNull;
        cudaError_t ce = cudaMemcpyAsync(d_seed, hs, sizeof hs, cudaMemcpyHostToDevice, s);
        // a pass starts from zero values, messages, rows and frontier
        if (ce == cudaSuccess) ce = cudaMemsetAsync(p.X, 0, 4 * V32, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(p.M, 0, 4 * V32, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(p.pdata, 0, 4ull * std::max<uint64_t>(g->npng_pad, 1) * kSeeds, s);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(p.bits, 0, 4 * (nw + 1), s);
        for (int i = 0; i < 3 && ce == cudaSuccess; ++i) ce = cudaMemsetAsync(pa[i], 0, g->k, s);
        if (ce != cudaSuccess) {
            status = fail(GPOP_ERR_CUDA, cudaGetErrorString(ce));
            break;
        }
        p.pact = pa[0]; p.pact_prev = pa[1]; p.pact_next = pa[2];
        k_binit<<<1, kSeeds, 0, s>>>(p);
        uint32_t it = 0;
        double hres[kSeeds] = {};
        bool conv = false;
        for (; it < o->max_iters; ++it) {
            p.epoch = ++epoch;
            timed(1, [&] { k_bscatter<<<std::min<uint32_t>(g->k, 8u * g->num_sms), kBThreads, 0, s>>>(p); });
            cudaMemsetAsync(p.counter, 0, 4, s);
            timed(4, [&] { k_bgather<<<g->num_sms, kBGThreads, gsmem, s>>>(p); });
            if (g->nmerge) timed(5, [&] { k_bmerge<<<std::min<uint32_t>(g->nmerge, 16u * g->num_sms), kBThreads, 0, s>>>(p); });
            cudaMemsetAsync(p.pact_next, 0, g->k, s);
            timed(3, [&] {
                k_bfilter<<<grid_f, kBThreads, 0, s>>>(p);
                k_bres<<<1, kSeeds, 0, s>>>(p, (uint32_t)grid_f);
            });
            ce = cudaMemcpyAsync(hres, p.res, sizeof hres, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce == cudaSuccess) ce = cudaGetLastError();
            if (ce != cudaSuccess) {
                status = fail(GPOP_ERR_CUDA, std::string("batched PPR: ") + cudaGetErrorString(ce));
                break;
            }
            uint8_t *old_prev = p.pact_prev;  // partitions active now become last iteration's
            p.pact_prev = p.pact;
            p.pact = p.pact_next;
            p.pact_next = old_prev;
            double mx = 0.0;
            for (uint32_t j = 0; j < n; ++j) mx = std::max(mx, hres[j]);
            total.residual = mx;
            if (o->tol_l1 > 0.0 && mx < o->tol_l1) {  // every seed's L1 change below the tolerance
                ++it;
                conv = true;
                break;
            }
        }
        if (status != GPOP_OK) break;
        total.iterations += it;
        total.converged &= conv ? 1 : 0;
        float *rows = out_values + (uint64_t)b0 * g->V;
        k_btranspose<<<(g->V + 31) / 32, dim3(32, 8), 0, s>>>(p.X, out_is_device ? rows : staging, g->V, n);
        if (!out_is_device) {
            ce = cudaMemcpyAsync(rows, staging, 4ull * n * g->V, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) status = fail(GPOP_ERR_CUDA, cudaGetErrorString(ce));
        }
    }
    cudaEventRecord(ev1, s);
    cudaEventSynchronize(ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    unsigned long long edges = 0;
    cudaMemcpy(&edges, p.edges, 8, cudaMemcpyDeviceToHost);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    cudaEventDestroy(kev[0]);
    cudaEventDestroy(kev[1]);
    if (status != GPOP_OK) return status;
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    total.device_ms = ms;
    total.edges_scattered = edges;
    total.pc_partition_steps = 0;
    if (stats) *stats = total;
    return GPOP_OK;
}
