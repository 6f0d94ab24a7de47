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
                    g->col_bins, g->png, g->pdata, g->row_png, g->cptr, g->cidx, g->cw,
                    g->scpair, g->sccnt, g->sub_cap, g->sub_task, g->row_sub, g->task_sub_ptr,
                    g->Ep, g->npng_p, g->nbins_p, g->gtask,
                    g->col_task, g->stask, g->pc_state, g->hidx, g->hw, g->hseg, g->hpart, g->task_hptr,
                    g->task_heavy};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete[] g->h_Ep;
    delete[] g->h_npng;
    *g = Graph();
}

namespace {

// RAII list of temporary device buffers released at scope exit.
struct Temps {
    std::vector<void *> ptrs;
    template <typename T>
    cudaError_t alloc(T **p, uint64_t count) {
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
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

// per sorted message j: bin boundary flags and histogram of messages / bins per row
__global__ void k_msg_bins(uint64_t nmsg, uint32_t shift, uint32_t k, const uint64_t *skey, uint32_t *newbin,
                           uint32_t *msgs_per_row, uint32_t *bins_per_row) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nmsg; j += stride) {
        uint64_t pk = skey[j] >> shift;
        uint32_t p = (uint32_t)(pk / k);
        bool nbf = (j == 0) || ((skey[j - 1] >> shift) != pk);
        newbin[j] = nbf;
        atomicAdd(&msgs_per_row[p], 1u);
        if (nbf) atomicAdd(&bins_per_row[p], 1u);
    }
}

__global__ void k_pad8(uint32_t k, const uint32_t *m, uint32_t *mp) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < k; p += gridDim.x * blockDim.x)
        mp[p] = (m[p] + kPngAlign - 1) / kPngAlign * kPngAlign;
}

// places every message in its padded PNG slot and records, per head edge, its slot and bin
__global__ void k_place_msgs(uint64_t nmsg, uint32_t shift, uint32_t k, const uint64_t *skey,
                             const uint32_t *shead, const uint32_t *binscan, const uint32_t *row_msg,
                             const uint32_t *row_png, uint16_t *png, uint32_t *slot_of_head,
                             uint32_t *bin_of_head, uint32_t *bin_q) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nmsg; j += stride) {
        uint64_t key = skey[j];
        uint64_t pk = key >> shift;
        uint32_t p = (uint32_t)(pk / k), q = (uint32_t)(pk % k);
        uint32_t slot = (uint32_t)j - row_msg[p] + row_png[p];
        png[slot] = (uint16_t)(key & ((1u << shift) - 1));
        uint32_t b = binscan[j] - 1;  // inclusive scan of new-bin flags
        slot_of_head[shead[j]] = slot;
        bin_of_head[shead[j]] = b;
        if (j == 0 || (skey[j - 1] >> shift) != pk) bin_q[b] = q;
    }
}

// every edge inherits the slot and bin of its message head
__global__ void k_edge_msg(uint64_t E, const uint32_t *head_of, const uint32_t *slot_of_head, const uint32_t *col,
                           uint64_t *ckey) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride)
        ckey[e] = ((uint64_t)col[e] << 32) | slot_of_head[head_of[e]];  // destination-major column lists
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

__global__ void k_indegree(uint64_t E, const uint32_t *col, uint32_t *indeg) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += stride)
        atomicAdd(&indeg[col[e]], 1u);
}

__global__ void k_unpack_csc(uint64_t E, uint32_t P, const uint64_t *key, uint32_t *cidx, uint16_t *cdst) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += stride) {
        uint64_t x = key[i];
        cidx[i] = (uint32_t)x;
        if (cdst) cdst[i] = (uint16_t)((x >> 32) & (P - 1));
    }
}

// splits the destination-sorted entries into light and heavy destinations
__global__ void k_heavy_flags(uint64_t E, const uint64_t *key, const uint32_t *indeg, uint32_t heavy, uint8_t *fl,
                              uint8_t *fh) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += stride) {
        bool h = indeg[(uint32_t)(key[i] >> 32)] > heavy;
        fl[i] = !h;
        fh[i] = h;
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
    return f(tmp, bytes);
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
    }

    // 3. messages: one per (source, destination partition), sorted by (p, q, source)
    uint8_t *head;
    uint64_t *mkey, *skey;
    uint32_t *head_idx, *shead, *d_nmsg;
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
    }
    g->npng = nmsg;

    // 4. bins, rows, padded PNG slots
    uint32_t *newbin, *binscan, *msgs_row, *row_msg, *msgs_row_pad;
    GPOP_CUDA_TRY(t.alloc(&newbin, nmsg));
    GPOP_CUDA_TRY(t.alloc(&binscan, nmsg));
    GPOP_CUDA_TRY(t.alloc(&msgs_row, (uint64_t)k + 1));
    GPOP_CUDA_TRY(t.alloc(&row_msg, (uint64_t)k + 1));
    GPOP_CUDA_TRY(t.alloc(&msgs_row_pad, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->nbins_p, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->npng_p, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->row_bin, (uint64_t)k + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->row_png, (uint64_t)k + 1));
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row, 0, 4ull * (k + 1), s));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->nbins_p, 0, 4ull * (k + 1), s));
    if (nmsg) {
        k_msg_bins<<<blocks_for(nmsg), kThreads, 0, s>>>(nmsg, shift, k, skey, newbin, msgs_row, g->nbins_p);
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::InclusiveSum(tmp, bytes, newbin, binscan, nmsg, s);
        }));
    }
    k_pad8<<<blocks_for(k), kThreads, 0, s>>>(k, msgs_row, msgs_row_pad);
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row_pad + k, 0, 4, s));
    GPOP_CUDA_TRY(cudaMemsetAsync(msgs_row + k, 0, 4, s));
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, msgs_row, row_msg, (uint64_t)k + 1, s);
    }));
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, msgs_row_pad, g->row_png, (uint64_t)k + 1, s);
    }));
    GPOP_CUDA_TRY(cudaMemcpyAsync(g->npng_p, msgs_row, 4ull * (k + 1), cudaMemcpyDeviceToDevice, s));
    GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
        return cub::DeviceScan::ExclusiveSum(tmp, bytes, g->nbins_p, g->row_bin, (uint64_t)k + 1, s);
    }));
    uint32_t h_npad = 0, h_nb = 0;
    GPOP_CUDA_TRY(cudaMemcpyAsync(&h_npad, g->row_png + k, 4, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(&h_nb, g->row_bin + k, 4, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    g->npng_pad = h_npad;
    g->nb = h_nb;

    GPOP_CUDA_TRY(dalloc(g, &g->png, g->npng_pad));
    GPOP_CUDA_TRY(dalloc(g, &g->pdata, g->npng_pad));
    GPOP_CUDA_TRY(dalloc(g, &g->bin_q, g->nb));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->png, 0, 2ull * std::max<uint64_t>(g->npng_pad, 1), s));
    GPOP_CUDA_TRY(cudaMemsetAsync(g->pdata, 0xFF, 4ull * std::max<uint64_t>(g->npng_pad, 1), s));
    uint32_t *slot_of_head, *bin_of_head;
    GPOP_CUDA_TRY(t.alloc(&slot_of_head, E));
    GPOP_CUDA_TRY(t.alloc(&bin_of_head, E));
    if (nmsg)
        k_place_msgs<<<blocks_for(nmsg), kThreads, 0, s>>>(nmsg, shift, k, skey, shead, binscan, row_msg, g->row_png,
                                                           g->png, slot_of_head, bin_of_head, g->bin_q);

    // 5. per-edge message slot (keys of the column lists)
    uint32_t *head_of;
    uint64_t *ckey;
    GPOP_CUDA_TRY(t.alloc(&head_of, E));
    GPOP_CUDA_TRY(t.alloc(&ckey, E));
    if (E) {
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::InclusiveScan(tmp, bytes, head_idx, head_of, MaxOp(), E, s);
        }));
        k_edge_msg<<<blocks_for(E), kThreads, 0, s>>>(E, head_of, slot_of_head, g->col, ckey);
    }

    // 6. destination lists grouped per destination vertex (column CSC over PNG slots).  A destination
    //    with more than kHeavy in-entries keeps its entries in a separate list cut into segments of at
    //    most kHeavySeg entries, reduced by their own warps so that no single task serialises a hub.
    GPOP_CUDA_TRY(dalloc(g, &g->cptr, (uint64_t)V + 1));
    GPOP_CUDA_TRY(dalloc(g, &g->cidx, E));
    if (g->weighted) GPOP_CUDA_TRY(dalloc(g, &g->cw, E));
    std::vector<uint32_t> hin(V);
    {
        uint32_t *indeg, *light;
        GPOP_CUDA_TRY(t.alloc(&indeg, (uint64_t)V + 1));
        GPOP_CUDA_TRY(t.alloc(&light, (uint64_t)V + 1));
        GPOP_CUDA_TRY(cudaMemsetAsync(indeg, 0, 4ull * (V + 1), s));
        if (E) k_indegree<<<blocks_for(E), kThreads, 0, s>>>(E, g->col, indeg);
        GPOP_CUDA_TRY(cudaMemcpyAsync(hin.data(), indeg, 4ull * V, cudaMemcpyDeviceToHost, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<uint32_t> hlight(V + 1, 0);
        uint64_t nheavy_entries = 0;
        for (uint32_t v = 0; v < V; ++v) {
            if (hin[v] > kHeavy) {
                g->h_hv.push_back(v);
                nheavy_entries += hin[v];
            } else {
                hlight[v] = hin[v];
            }
        }
        GPOP_CUDA_TRY(cudaMemcpyAsync(light, hlight.data(), 4ull * (V + 1), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
            return cub::DeviceScan::ExclusiveSum(tmp, bytes, light, g->cptr, (uint64_t)V + 1, s);
        }));
        g->nheavy = nheavy_entries;
        GPOP_CUDA_TRY(dalloc(g, &g->hidx, nheavy_entries));
        if (g->weighted) GPOP_CUDA_TRY(dalloc(g, &g->hw, nheavy_entries));
        if (E) {
            uint64_t *ck2, *ckl, *ckh;
            int32_t *cw2 = nullptr;
            uint8_t *fl, *fh;
            uint32_t *d_cnt;
            GPOP_CUDA_TRY(t.alloc(&ck2, E));
            GPOP_CUDA_TRY(t.alloc(&ckl, E));
            GPOP_CUDA_TRY(t.alloc(&ckh, nheavy_entries));
            GPOP_CUDA_TRY(t.alloc(&fl, E));
            GPOP_CUDA_TRY(t.alloc(&fh, E));
            GPOP_CUDA_TRY(t.alloc(&d_cnt, 2));
            int end_bit = 32 + bits_for(V);
            if (g->weighted) {
                GPOP_CUDA_TRY(t.alloc(&cw2, E));
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceRadixSort::SortPairs(tmp, bytes, ckey, ck2, g->w, cw2, E, 0, end_bit, s);
                }));
            } else {
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceRadixSort::SortKeys(tmp, bytes, ckey, ck2, E, 0, end_bit, s);
                }));
            }
            k_heavy_flags<<<blocks_for(E), kThreads, 0, s>>>(E, ck2, indeg, kHeavy, fl, fh);
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceSelect::Flagged(tmp, bytes, ck2, fl, ckl, d_cnt, (int64_t)E, s);
            }));
            GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                return cub::DeviceSelect::Flagged(tmp, bytes, ck2, fh, ckh, d_cnt + 1, (int64_t)E, s);
            }));
            if (g->weighted) {
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceSelect::Flagged(tmp, bytes, cw2, fl, g->cw, d_cnt, (int64_t)E, s);
                }));
                GPOP_CUDA_TRY(cub_run(t, [&](void *tmp, size_t &bytes) {
                    return cub::DeviceSelect::Flagged(tmp, bytes, cw2, fh, g->hw, d_cnt + 1, (int64_t)E, s);
                }));
            }
            uint64_t nlight = E - nheavy_entries;
            if (nlight) k_unpack_csc<<<blocks_for(nlight), kThreads, 0, s>>>(nlight, P, ckl, g->cidx, nullptr);
            if (nheavy_entries)
                k_unpack_csc<<<blocks_for(nheavy_entries), kThreads, 0, s>>>(nheavy_entries, P, ckh, g->hidx, nullptr);
        }
        // heavy destinations: contiguous entry ranges in destination order, cut into segments
        uint64_t off = 0;
        std::vector<uint4> segs;
        for (size_t i = 0; i < g->h_hv.size(); ++i) {
            uint32_t v = g->h_hv[i];
            g->h_hseg0.push_back((uint32_t)segs.size());
            for (uint64_t b = 0; b < hin[v]; b += kHeavySeg)
                segs.push_back(make_uint4(v, (uint32_t)(off + b), (uint32_t)std::min<uint64_t>(off + b + kHeavySeg, off + hin[v]), 0));
            off += hin[v];
        }
        g->h_hseg0.push_back((uint32_t)segs.size());
        g->nseg = (uint32_t)segs.size();
        GPOP_CUDA_TRY(dalloc(g, &g->hseg, g->nseg));
        GPOP_CUDA_TRY(dalloc(g, &g->hpart, g->nseg));
        if (g->nseg)
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->hseg, segs.data(), sizeof(uint4) * segs.size(), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    }

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

    // 8. per-partition statics
    GPOP_CUDA_TRY(dalloc(g, &g->Ep, (uint64_t)k + 1));
    k_part_edges<<<blocks_for(k), kThreads, 0, s>>>(k, V, shift, g->rowptr, g->Ep);
    std::vector<uint32_t> hEp(k), hnp(k), hnb(k), hrow_png(k + 1);
    GPOP_CUDA_TRY(cudaMemcpyAsync(hEp.data(), g->Ep, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hnp.data(), g->npng_p, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hnb.data(), g->nbins_p, 4ull * k, cudaMemcpyDeviceToHost, s));
    GPOP_CUDA_TRY(cudaMemcpyAsync(hrow_png.data(), g->row_png, 4ull * (k + 1), cudaMemcpyDeviceToHost, s));

    // 9. static gather tasks: destination ranges of <= kGatherWidth vertices, ~kGatherEntries in-entries
    uint32_t nblk = (V + 31) / 32;
    std::vector<uint32_t> hcnt(nblk, 0);  // light in-entries per block of 32 destinations
    for (uint32_t v = 0; v < V; ++v)
        if (hin[v] <= kHeavy) hcnt[v / 32] += hin[v];
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
    for (uint32_t q = 0; q < k; ++q) {
        col_task[q] = (uint32_t)gt.size();
        uint32_t b0 = (uint32_t)(((uint64_t)q << shift) / 32);
        uint32_t b1 = (uint32_t)std::min<uint64_t>((((uint64_t)q + 1) << shift) / 32, nblk);
        uint32_t base = b0;
        while (b0 < b1) {
            uint32_t e = 0, b = b0;
            while (b < b1 && (b - b0) < width_blocks && (b == b0 || e + hcnt[b] <= kGatherEntries)) e += hcnt[b++];
            gt.push_back(GatherTask{q, (b0 - base) * 32, (b - base) * 32, e});
            b0 = b;
        }
    }
    col_task[k] = (uint32_t)gt.size();
    g->ngt = (uint32_t)gt.size();
    // heavy destinations of every task: (local destination, first segment, segment count)
    {
        std::vector<uint32_t> thp(g->ngt + 1, 0);
        std::vector<uint4> th;
        size_t hi = 0;
        for (uint32_t ti = 0; ti < g->ngt; ++ti) {
            thp[ti] = (uint32_t)th.size();
            uint64_t lo = ((uint64_t)gt[ti].q << shift) + gt[ti].d0, up = ((uint64_t)gt[ti].q << shift) + gt[ti].d1;
            while (hi < g->h_hv.size() && g->h_hv[hi] < lo) ++hi;
            for (size_t j = hi; j < g->h_hv.size() && g->h_hv[j] < up; ++j)
                th.push_back(make_uint4((uint32_t)(g->h_hv[j] - ((uint64_t)gt[ti].q << shift) - gt[ti].d0),
                                        g->h_hseg0[j], g->h_hseg0[j + 1] - g->h_hseg0[j], 0));
        }
        thp[g->ngt] = (uint32_t)th.size();
        GPOP_CUDA_TRY(dalloc(g, &g->task_hptr, (uint64_t)g->ngt + 1));
        GPOP_CUDA_TRY(dalloc(g, &g->task_heavy, th.size()));
        GPOP_CUDA_TRY(cudaMemcpyAsync(g->task_hptr, thp.data(), 4ull * (g->ngt + 1), cudaMemcpyHostToDevice, s));
        if (!th.empty())
            GPOP_CUDA_TRY(cudaMemcpyAsync(g->task_heavy, th.data(), sizeof(uint4) * th.size(), cudaMemcpyHostToDevice, s));
        GPOP_CUDA_TRY(cudaStreamSynchronize(s));
    }
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
    if (P < 32 || P > 65536 || (P & (P - 1))) return fail(GPOP_ERR_INVALID_ARG, "partition_size must be a power of two in [32, 65536]");
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
    info->num_heavy_vertices = (uint32_t)g.h_hv.size();
    info->num_heavy_segments = g.nseg;
    info->num_heavy_entries = g.nheavy;
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
