// Internal declarations of the GB300 GPOP engine (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gpop.h"

namespace gpop {

// Reserved message value: a partition-centric message from an inactive source
// (and the "no message" state of a vertex).  As FP32 it is a NaN that no
// arithmetic of the applications produces; as uint32 it is above every vertex
// ID, distance and label.
constexpr uint32_t kNull = 0xFFFFFFFFu;
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kMsBfsWidth = 32;  // sources per multi-source BFS pass (bits of a 32-bit message)

constexpr int kPngAlign = 8;           // PNG rows padded to 8 entries (16-byte u16 vectors)
constexpr uint32_t kBinAlign = 8;      // every bin padded to 8 slots: 16-byte aligned bulk copies of bin runs (BF16)
constexpr uint32_t kGatherWidth = 4096;  // max destinations per gather task (smem accumulator)
constexpr uint64_t kGatherTaskMinEdges = 65536;  // in-edges a gather task may take before it is cut
constexpr uint32_t kGatherEntries = 32768;  // target in-entries per gather task
constexpr uint32_t kScatterChunk = 131072;  // PNG slots per PC scatter task (one staging of the partition's values)
constexpr uint32_t kMaxRowBins = 40960;     // SC scatter keeps one cursor per row bin in smem
constexpr uint32_t kPcBlock = 16384;        // messages staged in shared memory per PC gather block
constexpr uint32_t kPcTaskBlocks = 20;      // at most this many blocks per PC gather task (static smem per block)
constexpr uint32_t kPcGatherWarps = 23;     // consumer warps of the PC gather, one destination slice of each task each
constexpr uint32_t kPcPad = 16;             // each warp's entry range of a block is padded to a multiple of this
constexpr uint32_t kPcPadIdx = kPcBlock;    // block index of the padding entries (a value slot that holds NULL)
constexpr uint32_t kPcTaskMinEntries = 65536;  // PC gather tasks hold about max(this, E / (2 SMs)) entries
constexpr uint32_t kPcRound = 512;          // destination entries one gather warp folds per round

// A warp's entry range of a block is folded in rounds of kPcRound entries (the last one shorter, a
// multiple of kPcPad).  A round of n entries is shared by n / K lanes, K consecutive entries each:
__host__ __device__ constexpr uint32_t pc_round_k(uint32_t n) { return n <= 128 ? 4u : (n <= 256 ? 8u : 16u); }
// and is stored as K / 4 rows of 16-byte quads, row j holding the j-th quad of every lane, so that a warp
// reads one row with one coalesced 16-byte load per lane.  Position of entry m of a round of n entries:
__host__ __device__ constexpr uint32_t pc_round_pos(uint32_t m, uint32_t n) {
    return ((m % pc_round_k(n)) / 4 * (n / pc_round_k(n)) + m / pc_round_k(n)) * 4 + m % 4;
}
// Position of destination d in the gather's shared accumulator: bits 5-9 XORed into bits 0-4, a bijection
// on every aligned 32-word group that spreads the lanes of one fold step (destinations a near-constant
// stride apart) over distinct banks.  Destination entries carry the swizzled position.
__host__ __device__ constexpr uint32_t pc_swz(uint32_t d) { return d ^ ((d >> 5) & 31u); }

enum Mode : uint8_t { kModeNone = 0, kModeSC = 1, kModePC = 2 };
enum Action : uint8_t { kActSkip = 0, kActPC = 1, kActNull = 2 };

// Per-iteration control block written by the plan kernel and read by the host.
struct Control {
    unsigned long long frontier_v;   // sum of V_a entering the iteration
    unsigned long long frontier_e;   // sum of E_a
    double residual;                 // L1 change of the previous iteration (PR/PPR)
    double model_bytes;              // Sec. 3.2 bytes of this iteration's chosen modes
    uint32_t n_pc, n_sc, n_null;     // partitions per action
    uint32_t done;                   // 1 = stop before scattering this iteration
    uint32_t n_fallback;             // learned mode: partitions that fell back to Eq. (mode)
    uint32_t error;                  // device check flags
    uint32_t n_sc_units;             // SC scatter work units (split hub partitions count several)
    uint32_t pad;
    unsigned long long sc_v, sc_e;   // V_a and E_a of the partitions scattered in SC mode
};

// Static gather task: destinations [d0, d1) (local IDs) of column q, which have `entries` in-edges.
struct GatherTask {
    uint32_t q, d0, d1, entries;
};

// Static PC scatter task: PNG slots [beg, end) of partition p (padded row layout).
struct ScatterTask {
    uint32_t p, beg, end, first;  // first = 1 for the chunk that starts the row
};

struct Graph {
    uint32_t V = 0, P = 0, shift = 0, k = 0;
    uint64_t E = 0;
    int weighted = 0;
    uint64_t nb = 0, npng = 0, npng_pad = 0;
    uint32_t max_row_bins = 0;

    // CSR with rows sorted by destination
    uint32_t *rowptr = nullptr;   // V+1
    uint32_t *col = nullptr;      // E
    int32_t *w = nullptr;         // E or null
    uint16_t *esub = nullptr;     // E: index of the edge's SC bin within its bin row

    // bins bin[p][q] (non-empty), row-major
    uint32_t *row_bin = nullptr;  // k+1
    uint32_t *bin_q = nullptr;    // nb
    uint32_t *col_bin = nullptr;  // k+1
    uint32_t *col_bins = nullptr; // nb: bin ids per column, ascending p

    // PNG (Alg. 3) and PC data bins, padded rows
    uint16_t *png = nullptr;      // npng_pad: local source ID per message slot
    uint32_t *pdata = nullptr;    // npng_pad: message values
    uint32_t *row_png = nullptr;  // k+1: padded row offsets

    // PC gather blocks: each column's message sequence (bins (p, q), p ascending) cut into blocks of
    // kPcBlock messages, staged by runs; destination lists as (local destination << 16 | index in block)
    uint4 *pc_runs = nullptr;     // (row-major source slot, length, offset in block, block)
    uint32_t *pc_blk_run = nullptr;  // npcb+1: runs of each block
    uint32_t *pc_blk_nval = nullptr; // npcb: staged values of each block (a multiple of kBinAlign)
    uint2 *pc_blk_prange = nullptr;  // npcb: first and last source partition of each block's bins
    uint32_t *pc_blk_ent = nullptr;  // npcb+1: entries of each block
    uint4 *pc_task = nullptr;     // npct: (column, first block, end block, partial slot or kNull), largest first
    uint32_t *pc_tsp = nullptr;   // npct: first row of the task's blocks in pc_wsp
    uint32_t *pc_wsp = nullptr;   // per task block: kPcGatherWarps+1 entry offsets splitting its entries by
                                  // the task's destination slices (one slice per gather warp, the same in
                                  // every block of the task)
    uint32_t *col_ntask = nullptr;   // k: PC gather tasks of the column (0 = no PC in-edges)
    uint32_t *col_part0 = nullptr;   // k: first partial slot of a multi-task column
    uint32_t *pc_part = nullptr;  // npart x P partial results
    uint2 *pc_merge = nullptr;    // nmerge: (column, first destination) of each 1024-destination chunk of a
                                  // column split over several tasks (its partials are merged into pc_sum)
    uint32_t nmerge = 0;
    uint32_t *pe = nullptr;       // entries (swizzled accumulator position << 16 | index in block), sorted by
                                  // (block, destination, index); each warp range of a task block starts
                                  // 16-aligned, is padded to a multiple of kPcPad and is stored round by round
                                  // in lane-interleaved order (pc_round_pos)
    int32_t *pw = nullptr;        // null or weights aligned with pe (padding: 0)
    uint32_t npcb = 0, npct = 0, npart = 0;

    // SC bins, one per (source partition p, gather task t) with edges p -> t
    uint2 *scpair = nullptr;      // E: (local destination, value), regions of capacity edges(p, t)
    uint32_t *sccnt = nullptr;    // nsub: pairs written this iteration
    uint32_t *sub_cap = nullptr;  // nsub+1: region offsets
    uint32_t *sub_task = nullptr; // nsub: gather task of the bin
    uint32_t *row_sub = nullptr;  // k+1: bins of each source partition
    uint32_t *task_sub_ptr = nullptr;  // ngt+1: capacity of each task's fresh-bin list
    uint32_t nsub = 0, max_row_subs = 0;

    // per partition statics
    uint32_t *Ep = nullptr, *npng_p = nullptr, *nbins_p = nullptr;  // device, k each
    uint64_t *h_Ep = nullptr, *h_npng = nullptr;                      // host copies

    // tasks
    uint32_t ngt = 0, nst = 0;
    GatherTask *gtask = nullptr;  // ngt
    uint32_t *col_task = nullptr; // k+1
    ScatterTask *stask = nullptr; // nst

    // persistent run state (allocated lazily, reused across runs)
    uint8_t *pc_state = nullptr;  // k: row of pdata holds non-NULL values
    uint32_t epoch = 0;           // iteration stamp, never reused within the handle
    bool pdata_dirty = false;
    int pdata_fmt = 0;  // message format of the data rows: 0 FP32/u32, 1 BF16

    uint64_t device_bytes = 0;
    uint64_t fingerprint = 0;     // of the edge multiset with weights, V and E (checkpoints name their graph)
    std::vector<uint32_t> goff;   // graphs built as one disjoint union: first vertex of each (+ V at the end)
    int device = 0, num_sms = 0;
    void *run = nullptr;          // cached per-run buffers (engine.cu)
};

// error reporting (thread-local last error)
void set_error(const std::string &msg);
gpop_status fail(gpop_status st, const std::string &msg);

#define GPOP_CUDA_TRY(expr)                                                                       \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            return ::gpop::fail(GPOP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// device allocation helper tracked in Graph::device_bytes
template <typename T>
cudaError_t dalloc(Graph *g, T **p, uint64_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e == cudaSuccess) g->device_bytes += sizeof(T) * count;
    return e;
}

void free_graph(Graph *g);
void release_run_state(Graph *g);   // engine.cu
const float *selector_device_params();             // selector.cu: installed MLP parameters or null
const float *selector_device_params_transposed();  // the same with W1, W2 transposed (inference layout)

}  // namespace gpop

struct gpop_graph {
    gpop::Graph g;
};
