// Graph pre-processing (Sec. 3.1): index partitions, PNG layout of Alg. 3 with
// destination lists written once, SC bin capacities, gather/scatter task lists.
// Runs once per graph on the GPU; CUB radix sorts and scans are used as
// library primitives here (this step is outside the iteration hot path).
#include <cub/cub.cuh>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gpop_internal.cuh"

namespace gpop {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

gpop_status fail(gpop_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

void free_graph(Graph *g) {
    release_run_state(g);
    void *ptrs[] = {g->rowptr, g->col, g->w, g->esub, g->row_bin, g->bin_q, g->col_bin,
                    g->col_bins, g->png, g->pdata, g->row_png, g->pc_runs, g->pc_blk_run, g->pc_blk_nval, g->pc_blk_prange, g->pc_blk_ent,
                    g->pc_task, g->pc_tsp, g->pc_wsp, g->pc_merge, g->col_ntask, g->col_part0, g->pc_part, g->pe, g->pw,
                    g->scpair, g->sccnt, g->sub_cap, g->sub_task, g->row_sub, g->task_sub_ptr,
                    g->Ep, g->npng_p, g->nbins_p, g->gtask, g->col_task, g->stask, g->pc_state};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete[] g->h_Ep;
    delete[] g->h_npng;
    *g = Graph();
}

namespace {

// RAII list of temporary device buffers released at scope exit, or earlier by release() once a step no
// longer needs one (cudaFree waits for the work queued on the device, so no launch still reads it); the
// build's peak footprint is then a few steps' buffers instead of all of them.
struct Temps {
    std::vector<void *> ptrs;
    template <typename T>
    cudaError_t alloc(T **p, uint64_t count) {
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void *p) {
        for (size_t i = 0; i < ptrs.size(); ++i)
            if (ptrs[i] == p) {
                cudaFree(p);
                ptrs.erase(ptrs.begin() + (long)i);
                return;
            }
    }
    ~Temps() {
        for (void *p : ptrs) cudaFree(p);
    }
};

struct MaxOp {
    __host__ __device__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

constexpr int kThreads = 256;

inline unsigned blocks_for(uint64_t n, int per = kThreads) {
    uint64_t b = (n + per - 1) / per;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 1u << 22));
}

// --- validation --------------------------------------------------------------------------------

__global__ void k_validate(uint32_t V, uint64_t E, const uint64_t *rp, const uint32_t *col,
                           const int32_t *w, uint32_t *err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= V; i += stride) {
        if (i == 0 && rp[0] != 0) atomicOr(err, 1u);
        if (i == V && rp[V] != E) atomicOr(err, 2u);
        if (i < V && rp[i] > rp[i + 1]) atomicOr(err, 4u);
    }
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        if (col[e] >= V) atomicOr(err, 8u);
        if (w && w[e] < 0) atomicOr(err, 16u);
    }
}

__global__ void k_rowptr32(uint32_t V, const uint64_t *rp, uint32_t *out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= V; i += stride)
        out[i] = (uint32_t)rp[i];
}

// source vertex of every edge: largest u with rowptr[u] <= e
__global__ void k_edge_src(uint32_t V, uint64_t E, const uint32_t *rowptr, uint32_t *src) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        uint32_t lo = 0, hi = V;  // invariant rowptr[lo] <= e < rowptr[hi]
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (rowptr[mid] <= (uint32_t)e) lo = mid; else hi = mid;
        }
        src[e] = lo;
    }
}

__global__ void k_pack_src_dst(uint64_t E, const uint32_t *src, const uint32_t *col, uint64_t *key) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride)
        key[e] = ((uint64_t)src[e] << 32) | col[e];
}

__global__ void k_unpack_dst(uint64_t E, const uint64_t *key, uint32_t *col) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride)
        col[e] = (uint32_t)key[e];
}

// A message (Sec. 3.1.2) is one (source, destination partition) pair; its first
// edge in the destination-sorted row is the head.
__global__ void k_heads(uint64_t E, uint32_t shift, uint32_t k, const uint32_t *rowptr, const uint32_t *src,
                        const uint32_t *col, uint8_t *head, uint64_t *mkey, uint32_t *head_idx) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        uint32_t u = src[e], q = col[e] >> shift;
        bool h = (e == rowptr[u]) || ((col[e - 1] >> shift) != q);
        head[e] = h;
        uint32_t p = u >> shift, ul = u & ((1u << shift) - 1);
        mkey[e] = ((((uint64_t)p * k + q)) << shift) | ul;  // sort key (bin, local source)
        head_idx[e] = h ? (uint32_t)e : 0u;                 // for the max-scan
    }
}

// per sorted message j: does it start a new bin?
__global__ void k_msg_bins(uint64_t nmsg, uint32_t shift, const uint64_t *skey, uint32_t *newbin) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nmsg; j += stride)
        newbin[j] = (j == 0) || ((skey[j - 1] >> shift) != (skey[j] >> shift));
}

// Segment starts of keys sorted by seg(i) = (key[i] >> sh) / div, seg < nseg: start[s] = first index with
// seg >= s for s in [0, nseg], start[nseg] = n.  Each boundary writes the starts it crosses (no atomics).
__global__ void k_seg_starts(uint64_t n, const uint64_t *key, uint32_t sh, uint64_t div, uint32_t nseg,
                             uint32_t *start) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= n; i += stride) {
        const uint32_t hi = i < n ? (uint32_t)((key[i] >> sh) / div) : nseg;
        const uint32_t lo = i == 0 ? 0u : (uint32_t)((key[i - 1] >> sh) / div) + 1;
        for (uint32_t sg = lo; sg <= hi && sg <= nseg; ++sg) start[sg] = (uint32_t)i;
    }
}

// per row p: messages and bins, from the row's message range and the inclusive scan of new-bin flags
__global__ void k_row_counts(uint32_t k, const uint32_t *row_start, const uint32_t *binscan, uint32_t *msgs_row,
                             uint32_t *bins_row) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
        const uint32_t a = row_start[p], b = row_start[p + 1];
        msgs_row[p] = b - a;
        bins_row[p] = b > a ? binscan[b - 1] - (a > 0 ? binscan[a - 1] : 0u) : 0u;
    }
}

__global__ void k_pad8(uint32_t k, const uint32_t *m, uint32_t *mp) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
        mp[p] = (m[p] + kPngAlign - 1) / kPngAlign * kPngAlign;
}

// first message (sorted order), destination partition and source partition of every bin
__global__ void k_bin_starts(uint64_t nmsg, uint32_t shift, uint32_t k, const uint64_t *skey, const uint32_t *binscan,
                             uint32_t *bin_j0, uint32_t *bin_q, uint32_t *bin_p) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nmsg; j += stride) {
        uint64_t pk = skey[j] >> shift;
        if (j == 0 || (skey[j - 1] >> shift) != pk) {
            uint32_t b = binscan[j] - 1;
            bin_j0[b] = (uint32_t)j;
            bin_q[b] = (uint32_t)(pk % k);
            bin_p[b] = (uint32_t)(pk / k);
        }
    }
}

// every bin occupies its message count rounded up to kBinAlign slots of its PNG row (so that each bin,
// and each block of a column's message sequence, starts 16-byte aligned); per row, the padded length
__global__ void k_bin_pad(uint32_t nb, const uint32_t *bin_j0, const uint32_t *bin_p, uint32_t *cnt4,
                          uint32_t *row_len4) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        uint32_t c = (bin_j0[b + 1] - bin_j0[b] + kBinAlign - 1) / kBinAlign * kBinAlign;
        cnt4[b] = c;
        atomicAdd(&row_len4[bin_p[b]], c);
    }
}

// places every message in its PNG slot (row start + padded offset of its bin + rank in the bin) and
// records, per head edge, its slot and bin; bin_slot0 = slot of the bin's first message
__global__ void k_place_msgs(uint64_t nmsg, uint32_t shift, const uint64_t *skey, const uint32_t *shead,
                             const uint32_t *binscan, const uint32_t *bin_j0, const uint32_t *bin_p,
                             const uint32_t *binoff, const uint32_t *row_bin, const uint32_t *row_png, uint16_t *png,
                             uint32_t *slot_of_head, uint32_t *bin_of_head, uint32_t *bin_slot0) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nmsg; j += stride) {
        uint32_t b = binscan[j] - 1, p = bin_p[b];
        uint32_t slot = row_png[p] + (binoff[b] - binoff[row_bin[p]]) + ((uint32_t)j - bin_j0[b]);
        png[slot] = (uint16_t)(skey[j] & ((1u << shift) - 1));
        slot_of_head[shead[j]] = slot;
        bin_of_head[shead[j]] = b;
        if ((uint32_t)j == bin_j0[b]) bin_slot0[b] = slot;
    }
}

// key of every PC in-entry: (gather block << 32) | (local destination << 16) | index in the block,
// where the message of edge e is the one of its head (same source, same destination partition)
__global__ void k_pc_keys(uint64_t E, uint32_t shift, uint32_t P, const uint32_t *head_of,
                          const uint32_t *slot_of_head, const uint32_t *bin_of_head, const uint32_t *col,
                          const uint32_t *bin_slot0, const uint32_t *bin_cseq0, const uint32_t *col_blk0,
                          uint64_t *key) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        uint32_t h = head_of[e], b = bin_of_head[h], v = col[e];
        uint32_t cseq = bin_cseq0[b] + (slot_of_head[h] - bin_slot0[b]);
        uint32_t blk = col_blk0[v >> shift] + cseq / kPcBlock;
        key[e] = ((uint64_t)blk << 32) | ((uint64_t)(v & (P - 1)) << 16) | (cseq % kPcBlock);
    }
}

__global__ void k_pc_unpack(uint64_t E, const uint64_t *key, uint32_t *pe) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += stride) pe[i] = (uint32_t)key[i];
}

// SC bins are (source partition p, gather task t) pairs: key (p << 32) | t per edge
__global__ void k_sub_keys(uint64_t E, uint32_t shift, const uint32_t *src, const uint32_t *col,
                           const uint32_t *task_of, uint64_t *key) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride)
        key[e] = ((uint64_t)(src[e] >> shift) << 32) | task_of[col[e]];
}

__global__ void k_sub_split(uint64_t nsub, const uint64_t *ukey, uint32_t *sub_task, uint32_t *row_hist,
                            uint32_t *task_hist) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nsub; s += stride) {
        uint32_t tsk = (uint32_t)ukey[s];
        sub_task[s] = tsk;
        atomicAdd(&row_hist[(uint32_t)(ukey[s] >> 32)], 1u);
        atomicAdd(&task_hist[tsk], 1u);
    }
}

// in-degree of every 32-vertex block of destinations (where the gather tasks are cut)
__global__ void k_block_indeg(uint64_t E, const uint32_t *col, uint32_t *cnt) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) atomicAdd(&cnt[col[e] >> 5], 1u);
}

// index of every edge's SC bin within its bin row (binary search of its task in the row)
__global__ void k_edge_sub(uint64_t E, uint32_t shift, const uint32_t *src, const uint32_t *col,
                           const uint32_t *task_of, const uint32_t *row_sub, const uint32_t *sub_task, uint16_t *esub) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        uint32_t p = src[e] >> shift, tsk = task_of[col[e]];
        uint32_t lo = row_sub[p], hi = row_sub[p + 1];  // sub_task[lo..hi) ascending, contains tsk
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (sub_task[mid] <= tsk) lo = mid; else hi = mid;
        }
        esub[e] = (uint16_t)(lo - row_sub[p]);
    }
}

// splitmix64's output function (Steele, Lea, Flood 2014): a bijective 64-bit mix
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
// Fingerprint of the graph for checkpoints: the sum (mod 2^64) over edges of a mixed (source, destination,
// weight) key, so it depends on the edge multiset only, not on the order of the sums
__global__ void k_fingerprint(uint64_t E, const uint32_t *src, const uint32_t *col, const int32_t *w,
                              unsigned long long *out) {
    unsigned long long acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride) {
        const uint64_t wt = w ? (uint32_t)w[e] : 0u;
        acc += mix64((((uint64_t)src[e] << 32) | col[e]) ^ mix64(wt + 0x9E3779B97F4A7C15ull));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// first entry of [l, h) (sorted by destination) whose destination is at least D
__device__ __forceinline__ uint32_t first_dest_at_least(const uint32_t *pe, uint32_t l, uint32_t h, uint32_t D) {
    while (l < h) {
        const uint32_t m = l + (h - l) / 2;
        if ((pe[m] >> 16) < D) l = m + 1; else h = m;
    }
    return l;
}

// Destination cuts of the PC gather's warps, one set per task: the w-th cut (w = 1 .. kPcGatherWarps - 1)
// of task t is the smallest destination D such that at least w / kPcGatherWarps of the task's entries (over
// all its blocks, rows [row0[t], row0[t + 1]) with entries [lo, hi) each, sorted by destination) go to
// destinations below D.  Warp w then owns destinations [D_w, D_w+1) in every block of the task, so that
// gather warps working on different blocks never touch one destination.
__global__ void k_task_cuts(uint32_t ntask, uint32_t P, const uint32_t *row0, const uint32_t *lo, const uint32_t *hi,
                            const uint32_t *pe, uint32_t *cut) {
    constexpr uint32_t kW = kPcGatherWarps;
    const uint64_t n = (uint64_t)ntask * (kW - 1), stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t t = (uint32_t)(i / (kW - 1)), w = (uint32_t)(i % (kW - 1)) + 1;
        uint64_t total = 0;
        for (uint32_t r = row0[t]; r < row0[t + 1]; ++r) total += hi[r] - lo[r];
        const uint64_t target = (total * w + kW - 1) / kW;
        uint32_t a = 0, b = P;  // smallest D in [0, P] with count(dest < D) >= target
        while (a < b) {
            const uint32_t D = a + (b - a) / 2;
            uint64_t c = 0;
            for (uint32_t r = row0[t]; r < row0[t + 1]; ++r) c += first_dest_at_least(pe, lo[r], hi[r], D) - lo[r];
            if (c >= target) b = D; else a = D + 1;
        }
        cut[i] = a;
    }
}

// Warp splits of the PC gather: for every task block (entries [lo, hi), sorted by destination) and w in
// 0..kPcGatherWarps, the first entry of warp w's destinations [D_w, D_w+1) under its task's cuts.
__global__ void k_warp_splits(uint32_t nrow, const uint32_t *lo, const uint32_t *hi, const uint32_t *row_task,
                              const uint32_t *cut, const uint32_t *pe, uint32_t *out) {
    constexpr uint32_t kSp = kPcGatherWarps + 1;
    uint64_t n = (uint64_t)nrow * kSp, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t r = (uint32_t)(i / kSp), w = (uint32_t)(i % kSp);
        const uint32_t l = lo[r], h = hi[r];
        uint32_t a = w == 0 ? l : h;
        if (w > 0 && w < kPcGatherWarps)
            a = first_dest_at_least(pe, l, h, cut[(uint64_t)row_task[r] * (kPcGatherWarps - 1) + w - 1]);
        out[i] = a;
    }
}

// Copies each warp range [old0, old0 + len) of the destination entries to new0, padded to a multiple of
// kPcPad with entries that repeat the range's last destination and point to the padding value slot
// (which holds the monoid identity in the gather).  The range is stored round by round in the gather's
// lane-interleaved order (pc_round_pos), and every entry's destination field becomes its swizzled
// accumulator position (pc_swz; destinations stay equal exactly when their positions are).
__global__ void k_pad_entries(uint32_t nrange, const uint32_t *old0, const uint32_t *len, const uint32_t *new0,
                              const uint32_t *pe, const int32_t *pw, uint32_t *pe2, int32_t *pw2) {
    for (uint32_t r = blockIdx.x; r < nrange; r += gridDim.x) {
        const uint32_t a = old0[r], L = len[r], b = new0[r];
        const uint32_t PL = (L + kPcPad - 1) / kPcPad * kPcPad;
        for (uint32_t i = threadIdx.x; i < PL; i += blockDim.x) {
            uint32_t v;
            int32_t w = 0;
            if (i < L) {
                v = pe[a + i];
                if (pw) w = pw[a + i];
            } else {
                v = (pe[a + L - 1] & 0xFFFF0000u) | kPcPadIdx;
            }
            v = (pc_swz(v >> 16) << 16) | (v & 0xFFFFu);
            const uint32_t r0 = i / kPcRound * kPcRound;
            const uint32_t o = r0 + pc_round_pos(i - r0, min(kPcRound, PL - r0));
            pe2[b + o] = v;
            if (pw2) pw2[b + o] = w;
        }
    }
}

__global__ void k_colbin_keys(uint64_t nb, uint32_t k, const uint32_t *bin_q, const uint32_t *row_bin,
                              uint64_t *key, uint32_t *val, uint32_t *bins_per_col) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < nb; b += stride) {
        // row of bin b: largest p with row_bin[p] <= b
        uint32_t lo = 0, hi = k;
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (row_bin[mid] <= (uint32_t)b) lo = mid; else hi = mid;
        }
        key[b] = (uint64_t)bin_q[b] * k + lo;
        val[b] = (uint32_t)b;
        atomicAdd(&bins_per_col[bin_q[b]], 1u);
    }
}

__global__ void k_part_edges(uint32_t k, uint32_t V, uint32_t shift, const uint32_t *rowptr, uint32_t *Ep) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x) {
        uint64_t a = (uint64_t)p << shift, b = (uint64_t)(p + 1) << shift;
        if (b > V) b = V;
        Ep[p] = rowptr[b] - rowptr[a];
    }
}

template <typename F>
cudaError_t cub_run(Temps &t, F f) {
    size_t bytes = 0;
    cudaError_t e = f(nullptr, bytes);
    if (e != cudaSuccess) return e;
    void *tmp = nullptr;
    e = t.alloc((char **)&tmp, bytes);
    if (e != cudaSuccess) return e;
    e = f(tmp, bytes);
    t.release(tmp);
    return e;
}

int bits_for(uint64_t x) {  // number of bits to represent values < x
    int b = 0;
    while (b < 64 && (1ull << b) < x) ++b;
    return std::max(b, 1);
}

}  // namespace

static gpop_status build_impl(Graph *g, uint32_t V, uint64_t E, const uint64_t *row_ptr, const uint32_t *col,
                              const int32_t *weights, uint32_t P, int mem_is_device, cudaStream_t s) {
    GPOP_CUDA_TRY(cudaGetDevice(&g->device));
    GPOP_CUDA_TRY(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    g->V = V;
    g->E = E;
    g->P = P;
    g->shift = 0;
    while ((1u << g->shift) < P) ++g->shift;
    g->k = (uint32_t)(((uint64_t)V + P - 1) / P);
    g->weighted = weights != nullptr;
    const uint32_t k = g->k, shift = g->shift;
    Temps t;

    // 1. inputs on the device
    const uint64_t *d_rp = row_ptr;
    const uint32_t *d_col = col;
    const int32_t *d_w = weights;
    if (!mem_is_device) {
        uint64_t *a; uint32_t *b; int32_t *c = nullptr;
        GPOP_CUDA_TRY(t.alloc(&a, (uint64_t)V + 1));
        GPOP_CUDA_TRY(t.alloc(&b, E));
        GPOP_CUDA_TRY(cudaMemcpyAsync(a, row_ptr, sizeof(uint64_t) * (V + 1), cudaMemcpyHostToDevice, s));
        if (E) GPOP_CUDA_TRY(cudaMemcpyAsync(b, col, sizeof(uint32_t) * E, cudaMemcpyHostToDevice, s));
        if (weights) {
            GPOP_CUDA_TRY(t.alloc(&c, E));
            if (E) GPOP_CUDA_TRY(cudaMemcpyAsync(c, weights, sizeof(int32_t) * E, cudaMemcpyHostToDevice, s));
        }
        d_rp = a; d_col = b; d_w = c;
    }
    {
        uint32_t *d_err;
        GPOP_CUDA_TRY(t.alloc(&d_err, 1));
        GPOP_CUDA_TRY(cudaMemsetAsync(d_err, 0, 4, s));
        k_validate<<<blocks_for(std::max<uint64_t>(E, V + 1ull)), kThreads, 0, s>>>(V, E, d_rp, d_col, d_w, d_err);
        uint32_t herr = 0;
        GPOP_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        if (herr) {
            char buf[200];
            snprintf(buf, sizeof buf, "malformed CSR (flags 0x%x: 1 row_ptr[0]!=0, 2 row_ptr[V]!=E, 4 decreasing "
                     "row_ptr, 8 col>=V, 16 negative weight)", herr);
            return fail(GPOP_ERR_INVALID_ARG, buf);
        }
    }

    // 2. CSR with destination-sorted rows (u32 offsets)
    GPOP_CUDA_TRY(dalloc(g, &g->rowptr, (uint64_t)V + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->col, E));
    if (g->weighted) GPOP_CUDA_TRY(dalloc(g, &g->w, E));
    k_rowptr32<<<blocks_for(V + 1ull), kThreads, 0, s>>>(V, d_rp, g->rowptr);
    uint32_t *src;
    GPOP_CUDA_TRY(t.alloc(&src, E));
    if (E) {
        k_edge_src<<<blocks_for(E), kThreads, 0, s>>>(V, E, g->rowptr, src);
        uint64_t *k0, *k1;
        GPOP_CUDA_TRY(t.alloc(&k0, E));
        GPOP_CUDA_TRY(t.alloc(&k1, E));
        k_pack_src_dst<<<blocks_for(E), kThreads, 0, s>>>(E, src, d_col, k0);
        int end_bit = 32 + bits_for(V);
        if (g->weighted) {
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceRadixSort::SortPairs(tmp, bytes, k0, k1, d_w, g->w, E, 0, end_bit, s);
            }));
        } else {
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceRadixSort::SortKeys(tmp, bytes, k0, k1, E, 0, end_bit, s);
            }));
        }
        k_unpack_dst<<<blocks_for(E), kThreads, 0, s>>>(E, k1, g->col);
        t.release(k0);
        t.release(k1);
    }
    {  // the graph's fingerprint (checkpoints of another graph are refused)
        unsigned long long *d_fp, h_fp = 0;
        GPOP_CUDA_TRY(t.alloc(&d_fp, 1));
        GPOP_CUDA_TRY(cudaMemsetAsync(d_fp, 0, 8, s));
        if (E) k_fingerprint<<<std::min<uint64_t>(blocks_for(E), 8ull * g->num_sms), kThreads, 0, s>>>(E, src, g->col, g->w, d_fp);
        GPOP_CUDA_TRY(cudaMemcpyAsync(&h_fp, d_fp, 8, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        g->fingerprint = h_fp ^ ((uint64_t)V << 32) ^ (E * 0x9E3779B97F4A7C15ull) ^ (uint64_t)g->weighted;
    }

    // 3. messages: one per (source, destination partition), sorted by (p, q, source)
    uint8_t *head;
    uint64_t *mkey, *skey = nullptr;
    uint32_t *head_idx, *shead = nullptr, *d_nmsg;
    GPOP_CUDA_TRY(t.alloc(&head, E));
    GPOP_CUDA_TRY(t.alloc(&mkey, E));
    GPOP_CUDA_TRY(t.alloc(&head_idx, E));
    GPOP_CUDA_TRY(t.alloc(&d_nmsg, 1));
    GPOP_CUDA_TRY(cudaMemsetAsync(d_nmsg, 0, 4, s));
    uint64_t nmsg = 0;
    if (E) {
        k_heads<<<blocks_for(E), kThreads, 0, s>>>(E, shift, k, g->rowptr, src, g->col, head, mkey, head_idx);
        uint64_t *hkey;
        uint32_t *hidx;
        GPOP_CUDA_TRY(t.alloc(&hkey, E));
        GPOP_CUDA_TRY(t.alloc(&hidx, E));
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceSelect::Flagged(tmp, bytes, mkey, head, hkey, d_nmsg, (int64_t)E, s);
        }));
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceSelect::Flagged(tmp, bytes, head_idx, head, hidx, d_nmsg, (int64_t)E, s);
        }));
        t.release(mkey);
        uint32_t h_nmsg = 0;
        GPOP_CUDA_TRY(cudaMemcpyAsync(&h_nmsg, d_nmsg, 4, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        nmsg = h_nmsg;
        GPOP_CUDA_TRY(t.alloc(&skey, nmsg));
        GPOP_CUDA_TRY(t.alloc(&shead, nmsg));
        int end_bit = bits_for((uint64_t)k * k) + (int)shift;
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceRadixSort::SortPairs(tmp, bytes, hkey, skey, hidx, shead, nmsg, 0, end_bit, s);
        }));
        t.release(hkey);
        t.release(hidx);
    }
    t.release(head);
    g->npng = nmsg;

    // 4. bins, rows, padded PNG slots
    uint32_t *newbin, *binscan, *msgs_row, *msgs_row_pad, *row_start;
    GPOP_CUDA_TRY(t.alloc(&row_start, (uint64_t)k + 1));
    GPOP_CUDA_TRY(t.alloc(&newbin, nmsg));
    GPOP_CUDA_TRY(t.alloc(&binscan, nmsg));
    GPOP_CUDA_TRY(t.alloc(&msgs_row, (uint64_t)k + 1));
    GPOP_CUDA_TRY(t.alloc(&msgs_row_pad, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->nbins_p, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->npng_p, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->row_bin, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->row_png, (uint64_t)k + 1));
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row, 0, 4ull * (k + 1), s));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->nbins_p, 0, 4ull * (k + 1), s));
    if (nmsg) {
        k_msg_bins<<<blocks_for(nmsg), kThreads, 0, s>>>(nmsg, shift, skey, newbin);
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::InclusiveSum(tmp, bytes, newbin, binscan, nmsg, s);
        }));
    }
    t.release(newbin);
    // messages are sorted by (row p, column q, source): row p = (key >> shift) / k
    k_seg_starts<<<blocks_for(nmsg + 1), kThreads, 0, s>>>(nmsg, skey, shift, k, k, row_start);
    k_row_counts<<<blocks_for(k), kThreads, 0, s>>>(k, row_start, binscan, msgs_row, g->nbins_p);
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row + k, 0, 4, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(g->npng_p, msgs_row, 4ull * (k + 1), cudaMemcpyDeviceToDevice, s));
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, g->nbins_p, g->row_bin, (uint64_t)k + 1, s);
    }));
    uint32_t h_nb = 0;
    GPOP_CUDA_TRY(cudaMemcpyAsync(&h_nb, g->row_bin + k, 4, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    g->nb = h_nb;
    // bins padded to kBinAlign slots, rows to kPngAlign
    uint32_t *bin_j0, *bin_p, *cnt4, *binoff, *row_len4;
    GPOP_CUDA_TRY(t.alloc(&bin_j0, g->nb + 1));
    GPOP_CUDA_TRY(t.alloc(&bin_p, g->nb + 1));
    GPOP_CUDA_TRY(t.alloc(&cnt4, g->nb + 1));
    GPOP_CUDA_TRY(t.alloc(&binoff, g->nb + 1));
    GPOP_CUDA_TRY(t.alloc(&row_len4, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->bin_q, g->nb));
    GPOP_CUDA_TRY(cudaMemsetAsync(row_len4, 0, 4ull * (k + 1), s));
    const uint32_t nmsg32 = (uint32_t)nmsg;  // messages <= edges < 2^32
    GPOP_CUDA_TRY(cudaMemcpyAsync(bin_j0 + g->nb, &nmsg32, 4, cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(cnt4 + g->nb, 0, 4, s));
    if (nmsg) {
        k_bin_starts<<<blocks_for(nmsg), kThreads, 0, s>>>(nmsg, shift, k, skey, binscan, bin_j0, g->bin_q, bin_p);
        k_bin_pad<<<blocks_for(g->nb), kThreads, 0, s>>>((uint32_t)g->nb, bin_j0, bin_p, cnt4, row_len4);
    }
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, cnt4, binoff, g->nb + 1, s);
    }));
    k_pad8<<<blocks_for(k), kThreads, 0, s>>>(k, row_len4, msgs_row_pad);
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row_pad + k, 0, 4, s));
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, msgs_row_pad, g->row_png, (uint64_t)k + 1, s);
    }));
    uint32_t h_npad = 0;
    GPOP_CUDA_TRY(cudaMemcpyAsync(&h_npad, g->row_png + k, 4, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    g->npng_pad = h_npad;

    GPOP_CUDA_TRY(dalloc(g, &g->png, g->npng_pad));
    GPOP_CUDA_TRY(dalloc(g, &g->pdata, g->npng_pad));
    // padding slots keep local source 0: their values are staged but no entry refers to them
    GPOP_CUDA_TRY(cudaMemsetAsync(g->png, 0, 2ull * std::max<uint64_t>(g->npng_pad, 1), s));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->pdata, 0xFF, 4ull * std::max<uint64_t>(g->npng_pad, 1), s));
    uint32_t *slot_of_head, *bin_of_head, *bin_slot0;
    GPOP_CUDA_TRY(t.alloc(&slot_of_head, E));
    GPOP_CUDA_TRY(t.alloc(&bin_of_head, E));
    GPOP_CUDA_TRY(t.alloc(&bin_slot0, g->nb + 1));
    if (nmsg)
        k_place_msgs<<<blocks_for(nmsg), kThreads, 0, s>>>(nmsg, shift, skey, shead, binscan, bin_j0, bin_p, binoff,
                                                           g->row_bin, g->row_png, g->png, slot_of_head, bin_of_head,
                                                           bin_slot0);
    t.release(skey);
    t.release(shead);
    t.release(binscan);

    // 5. message head of every edge (its first edge to the same destination partition)
    uint32_t *head_of;
    GPOP_CUDA_TRY(t.alloc(&head_of, E));
    if (E) {
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::InclusiveScan(tmp, bytes, head_idx, head_of, MaxOp(), E, s);
        }));
    }
    t.release(head_idx);

    // 7. bins per column in ascending source partition
    GPOP_CUDA_TRY(dalloc(g, &g->col_bins, g->nb));
    GPOP_CUDA_TRY(dalloc(g, &g->col_bin, (uint64_t)k + 1));
    {
        uint64_t *bk, *bk2;
        uint32_t *bv, *bpc;
        GPOP_CUDA_TRY(t.alloc(&bk, g->nb));
        GPOP_CUDA_TRY(t.alloc(&bk2, g->nb));
        GPOP_CUDA_TRY(t.alloc(&bv, g->nb));
        GPOP_CUDA_TRY(t.alloc(&bpc, (uint64_t)k + 1));
        GPOP_CUDA_TRY(cudaMemsetAsync(bpc, 0, 4ull * (k + 1), s));
        if (g->nb) {
            k_colbin_keys<<<blocks_for(g->nb), kThreads, 0, s>>>(g->nb, k, g->bin_q, g->row_bin, bk, bv, bpc);
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceRadixSort::SortPairs(tmp, bytes, bk, bk2, bv, g->col_bins, g->nb, 0,
                                                       bits_for((uint64_t)k * k), s);
            }));
        }
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, bpc, g->col_bin, (uint64_t)k + 1, s);
        }));
    }

    // 6. PC gather blocks.  The messages of column q (its bins (p, q), p ascending, each bin's
    //    messages in source order) form the column sequence; it is cut into blocks of kPcBlock messages
    //    that the gather stages in shared memory by coalesced copies of bin runs ("runs": row-major
    //    source offset, length, offset in the block).  Every PC in-entry becomes a 4-byte word
    //    (local destination << 16 | index in its block), sorted by (block, destination, index).
    //    Gather tasks cover consecutive entries of one column: about max(kPcTaskMinEntries, E / (2 x
    //    SMs)) entries and at most kPcTaskBlocks blocks each, a block's entries split over several
    //    tasks when it is larger; a column with several tasks leaves one partial vector per task,
    //    merged in column order by the filter.  Tasks are listed largest first.
    {
        const uint32_t nb = (uint32_t)g->nb;
        std::vector<uint32_t> hj0(nb + 1), hslot0(nb), hcolbins(nb), hcolbin(k + 1), hbinp(nb);
        if (nb) {
            GPOP_CUDA_TRY(cudaMemcpyAsync(hbinp.data(), bin_p, 4ull * nb, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaMemcpyAsync(hj0.data(), bin_j0, 4ull * nb, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaMemcpyAsync(hslot0.data(), bin_slot0, 4ull * nb, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaMemcpyAsync(hcolbins.data(), g->col_bins, 4ull * nb, cudaMemcpyDeviceToHost, s));
        }
        GPOP_CUDA_TRY(cudaMemcpyAsync(hcolbin.data(), g->col_bin, 4ull * (k + 1), cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        hj0[nb] = (uint32_t)nmsg;
        std::vector<uint32_t> cseq0(nb + 1, 0), col_blk0(k + 1, 0);
        std::vector<uint4> runs;
        std::vector<uint32_t> blk_nval;  // staged values (padded messages) of every block
        std::vector<uint2> blk_prange;   // source partitions of every block's bins (first, last)
        uint32_t nblocks = 0;
        for (uint32_t q = 0; q < k; ++q) {
            col_blk0[q] = nblocks;
            uint64_t cs = 0;
            for (uint32_t i = hcolbin[q]; i < hcolbin[q + 1]; ++i) {
                const uint32_t b = hcolbins[i];
                const uint32_t cnt = (hj0[b + 1] - hj0[b] + kBinAlign - 1) / kBinAlign * kBinAlign;  // padded bin
                cseq0[b] = (uint32_t)cs;
                uint32_t done = 0;
                while (done < cnt) {  // split the bin's run at block boundaries
                    uint64_t pos = cs + done;
                    uint32_t piece = (uint32_t)std::min<uint64_t>(cnt - done, kPcBlock - pos % kPcBlock);
                    const uint32_t blk = nblocks + (uint32_t)(pos / kPcBlock);
                    runs.push_back(make_uint4(hslot0[b] + done, piece, (uint32_t)(pos % kPcBlock), blk));
                    if (blk >= blk_prange.size()) blk_prange.push_back(make_uint2(hbinp[b], hbinp[b]));
                    else blk_prange[blk].y = hbinp[b];  // bins of a column come in ascending source order
                    done += piece;
                }
                cs += cnt;
            }
            for (uint64_t j = 0; j < cs; j += kPcBlock) blk_nval.push_back((uint32_t)std::min<uint64_t>(kPcBlock, cs - j));
            nblocks += (uint32_t)((cs + kPcBlock - 1) / kPcBlock);
        }
        col_blk0[k] = nblocks;
        std::vector<uint32_t> blk_run0(nblocks + 1, (uint32_t)runs.size());
        for (size_t r = runs.size(); r-- > 0;) blk_run0[runs[r].w] = (uint32_t)r;
        for (uint32_t bl = nblocks; bl-- > 0;)  // blocks without runs (none in practice) take the next start
            if (blk_run0[bl] > blk_run0[bl + 1]) blk_run0[bl] = blk_run0[bl + 1];
        g->npcb = nblocks;
        GPOP_CUDA_TRY(dalloc(g, &g->pc_runs, runs.size()));
        GPOP_CUDA_TRY(dalloc(g, &g->pc_blk_run, (uint64_t)nblocks + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->pc_blk_ent, (uint64_t)nblocks + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->col_ntask, k));
        GPOP_CUDA_TRY(dalloc(g, &g->col_part0, k));
        // +4: the gather copies entry ranges as whole aligned 16-byte words
        GPOP_CUDA_TRY(dalloc(g, &g->pe, E + 4));
        if (g->weighted) GPOP_CUDA_TRY(dalloc(g, &g->pw, E + 4));
        if (!runs.empty())
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_runs, runs.data(), sizeof(uint4) * runs.size(), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_blk_run, blk_run0.data(), 4ull * (nblocks + 1), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(dalloc(g, &g->pc_blk_nval, (uint64_t)nblocks + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->pc_blk_prange, (uint64_t)nblocks + 1));
        if (blk_prange.size() != nblocks) return fail(GPOP_ERR_CUDA, "PC block layout: a block without runs");
        if (nblocks)
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_blk_prange, blk_prange.data(), sizeof(uint2) * nblocks, cudaMemcpyHostToDevice, s));
        if (nblocks)
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_blk_nval, blk_nval.data(), 4ull * nblocks, cudaMemcpyHostToDevice, s));
        // entries: sort keys (block, local destination, index in block)
        uint32_t *d_cseq0, *d_colblk0;
        GPOP_CUDA_TRY(t.alloc(&d_cseq0, nb + 1));
        GPOP_CUDA_TRY(t.alloc(&d_colblk0, (uint64_t)k + 1));
        GPOP_CUDA_TRY(cudaMemcpyAsync(d_cseq0, cseq0.data(), 4ull * (nb + 1), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaMemcpyAsync(d_colblk0, col_blk0.data(), 4ull * (k + 1), cudaMemcpyHostToDevice, s));
        if (E) {
            uint64_t *pk, *pk2;
            GPOP_CUDA_TRY(t.alloc(&pk, E));
            GPOP_CUDA_TRY(t.alloc(&pk2, E));
            k_pc_keys<<<blocks_for(E), kThreads, 0, s>>>(E, shift, P, head_of, slot_of_head, bin_of_head, g->col,
                                                         bin_slot0, d_cseq0, d_colblk0, pk);
            t.release(head_of);
            t.release(slot_of_head);
            t.release(bin_of_head);
            int end_bit = 32 + bits_for((uint64_t)nblocks + 1);
            if (g->weighted) {
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceRadixSort::SortPairs(tmp, bytes, pk, pk2, g->w, g->pw, E, 0, end_bit, s);
                }));
            } else {
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceRadixSort::SortKeys(tmp, bytes, pk, pk2, E, 0, end_bit, s);
                }));
            }
            k_pc_unpack<<<blocks_for(E), kThreads, 0, s>>>(E, pk2, g->pe);
            k_seg_starts<<<blocks_for(E + 1), kThreads, 0, s>>>(E, pk2, 32, 1, nblocks, g->pc_blk_ent);
            t.release(pk);
            t.release(pk2);
        } else {
            GPOP_CUDA_TRY(cudaMemsetAsync(g->pc_blk_ent, 0, 4ull * (nblocks + 1), s));
        }
        std::vector<uint32_t> hbe(nblocks + 1);
        GPOP_CUDA_TRY(cudaMemcpyAsync(hbe.data(), g->pc_blk_ent, 4ull * (nblocks + 1), cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));

        // gather tasks over each column's entries
        const uint64_t target = std::max<uint64_t>(kPcTaskMinEntries, E / (2ull * (uint64_t)std::max(1, g->num_sms)));
        std::vector<uint4> ptasks;
        std::vector<uint2> prng;
        std::vector<uint32_t> col_ntask(k, 0), col_part0(k, 0);
        uint32_t nparts = 0;
        for (uint32_t q = 0; q < k; ++q) {
            const uint32_t b_end = col_blk0[q + 1];
            uint32_t b = col_blk0[q];
            uint64_t pos = hbe[b];
            const uint64_t end = hbe[b_end];
            const size_t first_task = ptasks.size();
            for (;;) {
                while (b < b_end && pos >= hbe[b + 1]) ++b;  // skip exhausted blocks
                if (b == b_end || pos >= end) break;
                const uint32_t tb = b;
                const uint64_t ea = pos;
                uint64_t cnt = 0;
                uint32_t tb_end;
                for (;;) {
                    const uint64_t avail = hbe[b + 1] - pos, room = target - cnt;
                    if (avail >= room) {  // task full; the block may continue in the next task
                        pos += room;
                        tb_end = b + 1;
                        break;
                    }
                    cnt += avail;
                    pos = hbe[b + 1];
                    ++b;
                    if (b - tb == kPcTaskBlocks || b == b_end) {
                        tb_end = b;
                        break;
                    }
                }
                ptasks.push_back(make_uint4(q, tb, tb_end, kNull));
                prng.push_back(make_uint2((uint32_t)ea, (uint32_t)pos));
                b = tb_end - 1;
            }
            const uint32_t ntq = (uint32_t)(ptasks.size() - first_task);
            col_ntask[q] = ntq;
            col_part0[q] = nparts;
            if (ntq > 1) {
                for (uint32_t j = 0; j < ntq; ++j) ptasks[first_task + j].w = nparts + j;
                nparts += ntq;
            }
        }
        // largest tasks first, so that the persistent CTAs finish together
        std::vector<uint32_t> order(ptasks.size());
        for (uint32_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            return prng[x].y - prng[x].x > prng[y].y - prng[y].x;
        });
        std::vector<uint4> stasks(ptasks.size());
        std::vector<uint2> srng(ptasks.size());
        for (size_t i = 0; i < order.size(); ++i) {
            stasks[i] = ptasks[order[i]];
            srng[i] = prng[order[i]];
        }
        // warp splits: per task block, kPcGatherWarps entry ranges of about equal size cut at
        // destination boundaries
        constexpr uint32_t kSp = kPcGatherWarps + 1;
        {
            std::vector<uint32_t> tsp(stasks.size() + 1), rlo, rhi, rtask;
            for (size_t ti = 0; ti < stasks.size(); ++ti) {
                tsp[ti] = (uint32_t)rlo.size();
                const uint4 tk = stasks[ti];
                for (uint32_t b = tk.y; b < tk.z; ++b) {
                    rlo.push_back(b == tk.y ? srng[ti].x : hbe[b]);
                    rhi.push_back(b + 1 == tk.z ? srng[ti].y : hbe[b + 1]);
                    rtask.push_back((uint32_t)ti);
                }
            }
            tsp[stasks.size()] = (uint32_t)rlo.size();
            const uint32_t nrow = (uint32_t)rlo.size(), ntask = (uint32_t)stasks.size();
            uint32_t *d_lo, *d_hi, *d_rtask, *d_row0, *d_cut;
            GPOP_CUDA_TRY(t.alloc(&d_lo, (uint64_t)nrow + 1));
            GPOP_CUDA_TRY(t.alloc(&d_hi, (uint64_t)nrow + 1));
            GPOP_CUDA_TRY(t.alloc(&d_rtask, (uint64_t)nrow + 1));
            GPOP_CUDA_TRY(t.alloc(&d_row0, (uint64_t)ntask + 1));
            GPOP_CUDA_TRY(t.alloc(&d_cut, (uint64_t)ntask * (kPcGatherWarps - 1) + 1));
            GPOP_CUDA_TRY(dalloc(g, &g->pc_wsp, (uint64_t)nrow * kSp + 1));
            GPOP_CUDA_TRY(dalloc(g, &g->pc_tsp, (uint64_t)ntask + 1));
            if (nrow) {
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_lo, rlo.data(), 4ull * nrow, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_hi, rhi.data(), 4ull * nrow, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_rtask, rtask.data(), 4ull * nrow, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_row0, tsp.data(), 4ull * (ntask + 1), cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_tsp, tsp.data(), 4ull * ntask, cudaMemcpyHostToDevice, s));
                k_task_cuts<<<blocks_for((uint64_t)ntask * (kPcGatherWarps - 1)), kThreads, 0, s>>>(
                    ntask, g->P, d_row0, d_lo, d_hi, g->pe, d_cut);
                k_warp_splits<<<blocks_for((uint64_t)nrow * kSp), kThreads, 0, s>>>(nrow, d_lo, d_hi, d_rtask, d_cut,
                                                                                    g->pe, g->pc_wsp);
            }
            // re-lay the entries so that every warp range starts 16-aligned and is padded to kPcPad
            std::vector<uint32_t> sp((size_t)nrow * kSp);
            if (nrow) GPOP_CUDA_TRY(cudaMemcpyAsync(sp.data(), g->pc_wsp, 4ull * nrow * kSp, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaStreamSynchronize(s));
            const uint32_t nrange = nrow * kPcGatherWarps;
            std::vector<uint32_t> old0(nrange), len(nrange), new0(nrange), nsp((size_t)nrow * kSp);
            uint64_t pos = 0;
            for (uint32_t r = 0; r < nrow; ++r) {
                for (uint32_t w = 0; w < kPcGatherWarps; ++w) {
                    const uint32_t i = r * kPcGatherWarps + w, a = sp[(size_t)r * kSp + w];
                    old0[i] = a;
                    len[i] = sp[(size_t)r * kSp + w + 1] - a;
                    new0[i] = (uint32_t)pos;
                    nsp[(size_t)r * kSp + w] = (uint32_t)pos;
                    pos += (len[i] + kPcPad - 1) / kPcPad * kPcPad;
                }
                nsp[(size_t)r * kSp + kPcGatherWarps] = (uint32_t)pos;
            }
            if (pos + kPcPad >= (1ull << 32)) return fail(GPOP_ERR_INVALID_ARG, "too many edges for the padded PC entry layout");
            uint32_t *d_old0, *d_len, *d_new0, *pe2 = nullptr;
            int32_t *pw2 = nullptr;
            GPOP_CUDA_TRY(t.alloc(&d_old0, (uint64_t)nrange + 1));
            GPOP_CUDA_TRY(t.alloc(&d_len, (uint64_t)nrange + 1));
            GPOP_CUDA_TRY(t.alloc(&d_new0, (uint64_t)nrange + 1));
            cudaError_t ae = cudaMalloc(&pe2, 4ull * (pos + 4));
            if (ae == cudaSuccess && g->weighted) {
                ae = cudaMalloc(&pw2, 4ull * (pos + 4));
                if (ae != cudaSuccess) cudaFree(pe2);
            }
            GPOP_CUDA_TRY(ae);
            g->device_bytes += 4ull * (pos + 4) * (g->weighted ? 2 : 1);
            if (nrange) {
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_old0, old0.data(), 4ull * nrange, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_len, len.data(), 4ull * nrange, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(d_new0, new0.data(), 4ull * nrange, cudaMemcpyHostToDevice, s));
                GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_wsp, nsp.data(), 4ull * nrow * kSp, cudaMemcpyHostToDevice, s));
                k_pad_entries<<<std::min<uint32_t>(nrange, 65535u), kThreads, 0, s>>>(nrange, d_old0, d_len, d_new0,
                                                                                    g->pe, g->pw, pe2, pw2);
            }
            GPOP_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(g->pe);
            g->device_bytes -= 4ull * (E + 4);
            g->pe = pe2;
            if (g->weighted) {
                cudaFree(g->pw);
                g->device_bytes -= 4ull * (E + 4);
                g->pw = pw2;
            }
        }
        // merge items: 1024-destination chunks of every column split over several tasks
        {
            std::vector<uint2> items;
            for (uint32_t q = 0; q < k; ++q)
                if (col_ntask[q] > 1) {
                    const uint32_t wq = (uint32_t)std::min<uint64_t>(P, V - ((uint64_t)q << shift));
                    for (uint32_t d0 = 0; d0 < wq; d0 += 1024) items.push_back(make_uint2(q, d0));
                }
            g->nmerge = (uint32_t)items.size();
            GPOP_CUDA_TRY(dalloc(g, &g->pc_merge, items.size()));
            if (!items.empty())
                GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_merge, items.data(), sizeof(uint2) * items.size(), cudaMemcpyHostToDevice, s));
        }
        g->npct = (uint32_t)stasks.size();
        g->npart = nparts;
        GPOP_CUDA_TRY(dalloc(g, &g->pc_task, stasks.size()));
        GPOP_CUDA_TRY(dalloc(g, &g->pc_part, (uint64_t)nparts * P));
        if (!stasks.empty()) {
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->pc_task, stasks.data(), sizeof(uint4) * stasks.size(), cudaMemcpyHostToDevice, s));
        }
        GPOP_CUDA_TRY(cudaMemcpyAsync(g->col_ntask, col_ntask.data(), 4ull * k, cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaMemcpyAsync(g->col_part0, col_part0.data(), 4ull * k, cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    }

    // 8. per-partition statics
    GPOP_CUDA_TRY(dalloc(g, &g->Ep, (uint64_t)k + 1));
    k_part_edges<<<blocks_for(k), kThreads, 0, s>>>(k, V, shift, g->rowptr, g->Ep);
    std::vector<uint32_t> hEp(k), hnp(k), hnb(k), hrow_png(k + 1);
    GPOP_CUDA_TRY(cudaMemcpyAsync(hEp.data(), g->Ep, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hnp.data(), g->npng_p, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hnb.data(), g->nbins_p, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hrow_png.data(), g->row_png, 4ull * (k + 1), cudaMemcpyDeviceToHost, s));

    // 9. static gather tasks: ranges of whole 32-vertex blocks of one column, at most kGatherWidth
    //    destinations and (unless one block alone has more) at most `tgt` in-edges, so that the SC pairs
    //    of a hub column, which one task folds alone, are spread over several
    uint32_t nblk = (V + 31) / 32;
    std::vector<uint32_t> hin(nblk);
    {
        uint32_t *d_in;
        GPOP_CUDA_TRY(t.alloc(&d_in, nblk));
        GPOP_CUDA_TRY(cudaMemsetAsync(d_in, 0, 4ull * nblk, s));
        if (E) k_block_indeg<<<blocks_for(E), kThreads, 0, s>>>(E, g->col, d_in);
        GPOP_CUDA_TRY(cudaMemcpyAsync(hin.data(), d_in, 4ull * nblk, cudaMemcpyDeviceToHost, s));
    }
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    g->h_Ep = new uint64_t[k];
    g->h_npng = new uint64_t[k];
    g->max_row_bins = 0;
    for (uint32_t p = 0; p < k; ++p) {
        g->h_Ep[p] = hEp[p];
        g->h_npng[p] = hnp[p];
        g->max_row_bins = std::max(g->max_row_bins, hnb[p]);
    }
    if (g->max_row_bins > kMaxRowBins)
        return fail(GPOP_ERR_INVALID_ARG, "a bin row has more non-empty bins than the SC scatter supports; "
                                          "use a larger partition size");
    std::vector<GatherTask> gt;
    std::vector<uint32_t> col_task(k + 1);
    const uint32_t width_blocks = std::min(P, kGatherWidth) / 32;
    const uint64_t tgt = std::max<uint64_t>(kGatherTaskMinEdges, E / (4ull * (uint64_t)std::max(1, g->num_sms)));
    for (uint32_t q = 0; q < k; ++q) {
        col_task[q] = (uint32_t)gt.size();
        uint32_t b0 = (uint32_t)(((uint64_t)q << shift) / 32);
        uint32_t b1 = (uint32_t)std::min<uint64_t>((((uint64_t)q + 1) << shift) / 32, nblk);
        uint32_t base = b0;
        while (b0 < b1) {
            uint32_t b = b0;
            uint64_t in = 0;
            while (b < b1 && b - b0 < width_blocks && (b == b0 || in + hin[b] <= tgt)) in += hin[b++];
            gt.push_back(GatherTask{q, (b0 - base) * 32, (b - base) * 32, (uint32_t)std::min<uint64_t>(in, 0xFFFFFFFFu)});
            b0 = b;
        }
    }
    col_task[k] = (uint32_t)gt.size();
    g->ngt = (uint32_t)gt.size();
    GPOP_CUDA_TRY(dalloc(g, &g->gtask, g->ngt));
    GPOP_CUDA_TRY(dalloc(g, &g->col_task, (uint64_t)k + 1));
    GPOP_CUDA_TRY(cudaMemcpyAsync(g->gtask, gt.data(), sizeof(GatherTask) * gt.size(), cudaMemcpyHostToDevice, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(g->col_task, col_task.data(), 4ull * (k + 1), cudaMemcpyHostToDevice, s));

    // 10. static PC scatter tasks: padded rows in chunks of kScatterChunk slots
    std::vector<ScatterTask> st;
    for (uint32_t p = 0; p < k; ++p)
        for (uint32_t b = hrow_png[p]; b < hrow_png[p + 1]; b += kScatterChunk)
            st.push_back(ScatterTask{p, b, std::min(b + kScatterChunk, hrow_png[p + 1]), b == hrow_png[p]});
    g->nst = (uint32_t)st.size();
    GPOP_CUDA_TRY(dalloc(g, &g->stask, g->nst));
    if (g->nst)
        GPOP_CUDA_TRY(cudaMemcpyAsync(g->stask, st.data(), sizeof(ScatterTask) * st.size(), cudaMemcpyHostToDevice, s));

    // 11. SC bins at gather-task granularity: bin (p, t) receives the SC pairs from partition p to the
    //     destinations of gather task t (capacity = edges p -> t), so each gather task reads only its own
    {
        std::vector<uint32_t> task_of(V);
        for (uint32_t ti = 0; ti < g->ngt; ++ti) {
            uint64_t lo = ((uint64_t)gt[ti].q << shift) + gt[ti].d0;
            uint64_t hi = std::min<uint64_t>(((uint64_t)gt[ti].q << shift) + gt[ti].d1, V);
            for (uint64_t v = lo; v < hi; ++v) task_of[v] = ti;
        }
        uint32_t *d_task_of, *row_hist, *task_hist, *d_nsub;
        uint64_t *skey, *skey2, *ukey;
        uint32_t *counts;
        GPOP_CUDA_TRY(t.alloc(&d_task_of, V));
        GPOP_CUDA_TRY(t.alloc(&row_hist, (uint64_t)k + 1));
        GPOP_CUDA_TRY(t.alloc(&task_hist, (uint64_t)g->ngt + 1));
        GPOP_CUDA_TRY(t.alloc(&d_nsub, 1));
        GPOP_CUDA_TRY(t.alloc(&skey, E));
        GPOP_CUDA_TRY(t.alloc(&skey2, E));
        GPOP_CUDA_TRY(t.alloc(&ukey, E));
        GPOP_CUDA_TRY(t.alloc(&counts, E + 1));
        GPOP_CUDA_TRY(cudaMemcpyAsync(d_task_of, task_of.data(), 4ull * V, cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaMemsetAsync(row_hist, 0, 4ull * (k + 1), s));
        GPOP_CUDA_TRY(cudaMemsetAsync(task_hist, 0, 4ull * (g->ngt + 1), s));
        GPOP_CUDA_TRY(cudaMemsetAsync(d_nsub, 0, 4, s));
        uint32_t nsub = 0;
        if (E) {
            k_sub_keys<<<blocks_for(E), kThreads, 0, s>>>(E, shift, src, g->col, d_task_of, skey);
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceRadixSort::SortKeys(tmp, bytes, skey, skey2, E, 0, 32 + bits_for(k), s);
            }));
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceRunLengthEncode::Encode(tmp, bytes, skey2, ukey, counts, d_nsub, (int64_t)E, s);
            }));
            GPOP_CUDA_TRY(cudaMemcpyAsync(&nsub, d_nsub, 4, cudaMemcpyDeviceToHost, s));
            GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        }
        g->nsub = nsub;
        GPOP_CUDA_TRY(dalloc(g, &g->sub_cap, (uint64_t)nsub + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->sub_task, nsub));
        GPOP_CUDA_TRY(dalloc(g, &g->row_sub, (uint64_t)k + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->task_sub_ptr, (uint64_t)g->ngt + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->esub, E));
        GPOP_CUDA_TRY(cudaMemsetAsync(counts + nsub, 0, 4, s));
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, counts, g->sub_cap, (uint64_t)nsub + 1, s);
        }));
        if (nsub) k_sub_split<<<blocks_for(nsub), kThreads, 0, s>>>(nsub, ukey, g->sub_task, row_hist, task_hist);
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, row_hist, g->row_sub, (uint64_t)k + 1, s);
        }));
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, task_hist, g->task_sub_ptr, (uint64_t)g->ngt + 1, s);
        }));
        std::vector<uint32_t> hrow(k);
        GPOP_CUDA_TRY(cudaMemcpyAsync(hrow.data(), row_hist, 4ull * k, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        g->max_row_subs = 0;
        for (uint32_t p = 0; p < k; ++p) g->max_row_subs = std::max(g->max_row_subs, hrow[p]);
        if (g->max_row_subs > kMaxRowBins)
            return fail(GPOP_ERR_INVALID_ARG, "a partition sends SC messages to more gather tasks than the SC "
                                              "scatter supports; use a larger partition size");
        if (E) k_edge_sub<<<blocks_for(E), kThreads, 0, s>>>(E, shift, src, g->col, d_task_of, g->row_sub,
                                                             g->sub_task, g->esub);
    }
    GPOP_CUDA_TRY(dalloc(g, &g->scpair, E));
    GPOP_CUDA_TRY(dalloc(g, &g->sccnt, g->nsub));
    GPOP_CUDA_TRY(dalloc(g, &g->pc_state, k));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->pc_state, 0, k, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    GPOP_CUDA_TRY(cudaGetLastError());
    return GPOP_OK;
}

}  // namespace gpop

using namespace gpop;

extern "C" gpop_status gpop_graph_build(uint32_t num_vertices, uint64_t num_edges, const uint64_t *row_ptr,
                                        const uint32_t *col, const int32_t *weights, uint32_t partition_size,
                                        int mem_is_device, void *cuda_stream, gpop_graph **out) {
    set_error("");
    if (!out) return fail(GPOP_ERR_INVALID_ARG, "out is NULL");
    if (num_vertices == 0 || num_vertices >= (1u << 31)) return fail(GPOP_ERR_INVALID_ARG, "num_vertices out of range");
    if (num_edges >= (1ull << 32)) return fail(GPOP_ERR_INVALID_ARG, "num_edges must be < 2^32");
    if (!row_ptr || (num_edges && !col)) return fail(GPOP_ERR_INVALID_ARG, "row_ptr/col is NULL");
    uint32_t P = partition_size;
    if (P == 0) {
        P = 32;
        while (P < 16384 && P < num_vertices) P <<= 1;
    }
    if (P < 32 || P > 16384 || (P & (P - 1))) return fail(GPOP_ERR_INVALID_ARG, "partition_size must be a power of two in [32, 16384]");
    if (((uint64_t)num_vertices + P - 1) / P > 65536) return fail(GPOP_ERR_INVALID_ARG, "more than 65536 partitions");
    gpop_graph *h = new (std::nothrow) gpop_graph();
    if (!h) return fail(GPOP_ERR_OOM, "host allocation failed");
    gpop_status st = build_impl(&h->g, num_vertices, num_edges, row_ptr, col, weights, P, mem_is_device,
                                (cudaStream_t)cuda_stream);
    if (st != GPOP_OK) {
        cudaGetLastError();
        free_graph(&h->g);
        delete h;
        if (st == GPOP_ERR_CUDA && std::string(gpop_last_error()).find("out of memory") != std::string::npos)
            st = GPOP_ERR_OOM;
        return st;
    }
    *out = h;
    return GPOP_OK;
}

extern "C" gpop_status gpop_graph_build_union(uint32_t num_graphs, const uint32_t *num_vertices,
                                              const uint64_t *num_edges, const uint64_t *const *row_ptrs,
                                              const uint32_t *const *cols, const int32_t *const *weights,
                                              uint32_t partition_size, void *cuda_stream, gpop_graph **out) {
    set_error("");
    if (!out || !num_vertices || !num_edges || !row_ptrs || !cols) return fail(GPOP_ERR_INVALID_ARG, "NULL argument");
    if (num_graphs == 0) return fail(GPOP_ERR_INVALID_ARG, "no graphs");
    // the union's CSR: graph i's vertices follow graph i-1's, its edges shifted by its first vertex
    std::vector<uint32_t> goff(num_graphs + 1, 0);
    uint64_t V = 0, E = 0;
    for (uint32_t i = 0; i < num_graphs; ++i) {
        if (num_vertices[i] == 0) return fail(GPOP_ERR_INVALID_ARG, "a graph without vertices");
        if (!row_ptrs[i] || (num_edges[i] && !cols[i])) return fail(GPOP_ERR_INVALID_ARG, "a graph's row_ptr/col is NULL");
        if ((weights != nullptr) && !weights[i] && num_edges[i]) return fail(GPOP_ERR_INVALID_ARG, "weights for some graphs only");
        if (row_ptrs[i][0] != 0 || row_ptrs[i][num_vertices[i]] != num_edges[i])
            return fail(GPOP_ERR_INVALID_ARG, "a graph's row_ptr does not span its edges");
        goff[i] = (uint32_t)std::min<uint64_t>(V, 0xFFFFFFFFull);
        V += num_vertices[i];
        E += num_edges[i];
        if (V >= (1ull << 31)) return fail(GPOP_ERR_INVALID_ARG, "the union has 2^31 vertices or more");
        if (E >= (1ull << 32)) return fail(GPOP_ERR_INVALID_ARG, "the union has 2^32 edges or more");
    }
    goff[num_graphs] = (uint32_t)V;
    std::vector<uint64_t> rp(V + 1);
    std::vector<uint32_t> col(std::max<uint64_t>(E, 1));
    std::vector<int32_t> w(weights ? std::max<uint64_t>(E, 1) : 0);
    uint64_t eo = 0;
    for (uint32_t i = 0; i < num_graphs; ++i) {
        const uint32_t n = num_vertices[i], base = goff[i];
        for (uint32_t v = 0; v < n; ++v) rp[base + v] = eo + row_ptrs[i][v];
        for (uint64_t e = 0; e < num_edges[i]; ++e) {
            if (cols[i][e] >= n) return fail(GPOP_ERR_INVALID_ARG, "a destination outside its graph");
            col[eo + e] = base + cols[i][e];
            if (weights) w[eo + e] = weights[i][e];
        }
        eo += num_edges[i];
    }
    rp[V] = E;
    gpop_status st = gpop_graph_build((uint32_t)V, E, rp.data(), col.data(), weights ? w.data() : nullptr,
                                      partition_size, 0, cuda_stream, out);
    if (st == GPOP_OK) (*out)->g.goff = std::move(goff);
    return st;
}

extern "C" gpop_status gpop_graph_union_offsets(const gpop_graph *h, uint32_t *offsets, uint32_t *num_graphs) {
    if (!h || !num_graphs) return fail(GPOP_ERR_INVALID_ARG, "NULL argument");
    const uint32_t n = h->g.goff.empty() ? 0u : (uint32_t)h->g.goff.size() - 1;
    *num_graphs = n;
    if (offsets)
        for (uint32_t i = 0; i <= n && n; ++i) offsets[i] = h->g.goff[i];
    return GPOP_OK;
}

extern "C" gpop_status gpop_graph_get_info(const gpop_graph *h, gpop_graph_info *info) {
    if (!h || !info) return fail(GPOP_ERR_INVALID_ARG, "NULL argument");
    const Graph &g = h->g;
    memset(info, 0, sizeof *info);
    info->num_vertices = g.V;
    info->partition_size = g.P;
    info->num_partitions = g.k;
    info->weighted = (uint32_t)g.weighted;
    info->num_edges = g.E;
    info->num_bins = g.nb;
    info->num_png = g.npng;
    info->num_png_padded = g.npng_pad;
    info->num_gather_tasks = g.ngt;
    info->num_scatter_tasks = g.nst;
    info->max_row_bins = g.max_row_bins;
    info->device_bytes = g.device_bytes;
    info->num_pc_blocks = g.npcb;
    info->num_pc_tasks = g.npct;
    info->num_pc_partials = g.npart;
    return GPOP_OK;
}

extern "C" gpop_status gpop_graph_partition_stats(const gpop_graph *h, uint64_t *edges, uint64_t *png) {
    if (!h) return fail(GPOP_ERR_INVALID_ARG, "NULL graph");
    for (uint32_t p = 0; p < h->g.k; ++p) {
        if (edges) edges[p] = h->g.h_Ep[p];
        if (png) png[p] = h->g.h_npng[p];
    }
    return GPOP_OK;
}

extern "C" void gpop_graph_destroy(gpop_graph *h) {
    if (!h) return;
    free_graph(&h->g);
    delete h;
}

extern "C" const char *gpop_last_error(void) { return gpop::g_last_error.c_str(); }
