// gbx_internal.cuh -- internal declarations of the gbx library (not installed).
//
// Data model (all device memory):
//   * A "move program" is a list of levels; every level is one or two fused kernel
//     launches (copy ops, fold ops) whose ops are independent; levels run in order.
//   * A COPY op moves elements: its element space [0, nelem) is cut into segments,
//     each a run whose destination is contiguous; the source is contiguous or gathered
//     through a per-element int32 index (the pack-by-send-index-list step of the
//     neighbourhood exchange).  Standard forward = 1 copy op; locality forward =
//     {direct, gather} -> {node-pair block copy} -> {redistribute}.
//   * A FOLD op sums, for every output row, a fixed-order list of additive terms
//     (the reverse exchange); terms carry a group-start bit so that one row can fold
//     per-group partial sums (the node-blocked order).
//   * Tiles are GBX_TILE chunks (a chunk = one vector of `vec` bytes); every launch
//     uses blockDim * unroll == GBX_TILE, so ops of different patterns, element sizes and
//     vector widths share one grid (the batched launch).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gbx.h"

#include "gbx_device.cuh"

// ----------------------------------------------------------------------------- util
#define GBX_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) {                            \
            gbx_note_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return _e == cudaErrorMemoryAllocation ? GBX_ERR_NOMEM : GBX_ERR_CUDA; \
        }                                                   \
    } while (0)

#define GBX_TRY(expr)                  \
    do {                               \
        int _rc = (expr);              \
        if (_rc != GBX_SUCCESS) return _rc; \
    } while (0)

void gbx_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// NVTX range for the scope of a host call: setup stages, starts and (with graph=0) each
// phase's kernel launch get a name a profiler can attribute time to.  NVTX v3 is header-only:
// with no tool attached a push / pop is a call through a no-op function pointer.
struct GbxRange {
    explicit GbxRange(const char *name) { nvtxRangePushA(name); }
    ~GbxRange() { nvtxRangePop(); }
    GbxRange(const GbxRange &) = delete;
    GbxRange &operator=(const GbxRange &) = delete;
};
static inline int bitlen_u64(uint64_t x) { int n = 0; while (x) { n++; x >>= 1; } return n; }

// Device allocations owned by one object; freed together.
struct DevPool {
    std::vector<void *> ptrs;
    int64_t bytes = 0;
    int alloc(void **p, size_t n);   // GBX_SUCCESS / GBX_ERR_NOMEM
    template <typename T>
    int get(T **p, int64_t count) { return alloc(reinterpret_cast<void **>(p), (size_t)(count > 0 ? count : 1) * sizeof(T)); }
    void release();
    ~DevPool() { release(); }
};

// ------------------------------------------------------------------- primitives
// Exclusive scan of n int64 values into out[0..n]; out[n] receives the total.
int gbx_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st, DevPool &ws);
// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of the keys.
// On return *keys / *vals point at the sorted arrays (one of the two buffers given).
int gbx_sort_pairs(uint64_t **keys, int64_t **vals, uint64_t *keys_alt, int64_t *vals_alt,
                   int64_t n, int bits, cudaStream_t st, DevPool &ws);
int gbx_read_err(int *d_err, cudaStream_t st);   // syncs, returns first (lowest) code
int gbx_fill_i64(int64_t *p, int64_t v, int64_t n, cudaStream_t st);
int gbx_iota_i64(int64_t *p, int64_t n, cudaStream_t st);
int gbx_read_i64(const int64_t *d, int64_t *h, cudaStream_t st);

// ------------------------------------------------------------------ move kernels
// Kernels are specialised per vector width (copy) or (payload type, vector width)
// (fold); vec == 0 selects the generic kernel that dispatches per tile, used when one
// launch mixes ops of different widths (batched patterns).
int gbx_num_sms(void);
int gbx_effective_block(int vec, int block);
int gbx_occupancy(int kind, int dtype, int vec, int block, int flat);   // resident blocks per SM
// flat: 0 every op in segment form, 1 every op in flat form, 2 decided per op
cudaError_t gbx_launch_copy(const CopyDesc *const *ops, const int64_t *tile_prefix, int nops,
                            int64_t total_tiles, int vec, int flat, int block, int grid, cudaStream_t st);
// form 0: the fold kernel; 1: its stream form (records and terms staged in shared memory)
cudaError_t gbx_launch_fold(const FoldDesc *const *ops, const int64_t *tile_prefix, int nops,
                            int64_t total_tiles, int dtype, int vec, int block, int grid,
                            cudaStream_t st, int form);
int gbx_sfold_prepare(void);
// Per-tile metadata: first unit (element / row) of each tile and, for copy ops, the
// segment holding it (segs may be NULL for fold ops).
int gbx_build_tile_meta(const Seg *segs, int64_t nseg, int cpe, int64_t ntiles, int64_t *tile_seg,
                        int64_t *tile_e0, cudaStream_t st);

// ------------------------------------------------------------------------ objects
struct gbx_comm_s {
    int P, ppn, nnodes;
};

struct gbx_graph_s {
    gbx_comm_s *comm;
    int P, ppn, nnodes, device;
    int64_t E;
    DevPool mem;
    int *in_ptr, *sources, *out_ptr, *dests;  // library copies
    int *in_owner, *out_owner;                // rank owning each in / out edge
    int64_t *match_out;                       // out-edge -> in-edge
    int64_t *match_in;                        // in-edge -> out-edge
};

// One op of a move program, host side.
struct HostOp {
    int kind;        // 0 copy, 1 fold
    int level;
    int64_t units;   // elements (copy) or rows (fold)
    int max_vec;     // widest vector the alignment allows
    int min_vec;     // narrowest vector the kernel accepts (fold: the payload type)
    int block;       // tuned block size (block * unroll == GBX_TILE)
    int persistent;  // tuned grid: 1 = resident blocks only, 0 = one block per tile
    float tuned_ms;  // measured time of the tuned shape (0 if not tuned)
    int64_t algo_bytes;
    int64_t idx_len; // copy: entries of the index array; fold: number of terms
    CopyDesc cd;     // host copies of the descriptor
    FoldDesc fd;
    void *d_desc;           // device descriptor
    longlong2 *d_rec;       // fold: packed row records
    int64_t *d_tile_seg;    // copy: tile_seg storage sized for min_vec
    int64_t *d_tile_e0;     // tile_e0 storage sized for min_vec
    int32_t *d_flat_idx;    // copy: source element of every element when the flat form applies
    int64_t flat_dst0;
    int flat_ok;            // the flat form is available
    int flat_only;          // the op exists only in flat form (cd.flat is 1 or 3)
    int64_t algo_bytes_flat;
    int64_t algo_bytes_bulk;
    int64_t algo_bytes_seg;   // the segment form's
    int bulk_ok;            // every segment is contiguous on both sides and 16-byte aligned
    BulkTask *d_bulk;       // its pieces for the bulk form
    int64_t nbulk;
    int stream_ok;          // the flat form's index arrays are 16-byte aligned and padded: the
                            // stream forms (10 gather, 11 two-index) are available
    int sfold_ok;           // fold: records and terms aligned and padded, one payload class: the
                            // stream form of the fold is available
    int fold_form;          // fold: 0 the fold kernel, 1 its stream form (tuned)
    int scat_ok;            // two-index copy with the scatter form available
    ScatterPiece *d_scat;
    int64_t nscat;
    int64_t algo_bytes_scat;
    void **d_self;          // one-entry descriptor list for launching the op alone
    int64_t *d_self_prefix; // {0, ntiles}
};

// One kernel launch of a level.
struct LevelLaunch {
    int kind;
    int dtype;              // fold: payload type
    int vec;                // vector width of every op, or 0 when they differ
    int flat;               // copy: 0 / 1 when every op uses the segment / flat form, 2 mixed
    int block;
    int grid;
    int nops;
    int64_t total_tiles;
    int max_ctas;           // grid cap (0: none)
    const char *phase;      // NVTX name of the launch (a string literal)
    int one;                // copies: every op has one chunk per element (stream kernels specialise)
    void **d_ops;           // device array of descriptor pointers
    int64_t *d_prefix;      // device tile prefix (nops + 1)
};

struct Batch;

struct gbx_request_s {
    int device;
    int kind;                // 0 forward, 1 backward
    int algorithm;
    int use_graph, autotune, forced_vec, forced_block;
    int min_run;             // gathered runs of at least this many elements become contiguous (0 = off)
    int piece;               // > 0: copy ops run in source order, in pieces of at most this many elements
    int forced_flat;         // -1: the tuner chooses the flat form or segments; 0 / 1: forced
    int allow_flat;
    int no_combine;          // locality form: keep direct copies and redistribution apart
    int no_single_split;     // keep single-term fold rows in the fold
    int split_order;         // single-term rows as copies: 0 in row (destination) order, 1 in source order
    int check_dup;           // locality form: compare every deduplicated value's bytes with its representative's at init
    int allow_bulk;          // offer the bulk form to the autotuner where it applies
    int allow_stream;        // 0: no stream forms, 1: offered to the autotuner, 2: forced where they apply
    int forced_form;         // -1, or the one copy form the tuner times where an op offers it
    int max_ctas;            // cap on every launch's grid (0: none)
    int timeout_ms;
    int wait_limit;          // polls of the main waits of the bulk / scatter kernels
    // the request's status word: pinned host memory mapped into the device, written by its
    // kernels when a bounded wait gives up (1) or a piece fails its check (2), read and
    // cleared by gbx_test / gbx_wait
    int *status_host;
    int *status_dev;
    gbx_graph_s *graph;
    gbx_request_s *forward;  // backward: its forward request
    gbx_graph_s *owned_graph;  // graph built for this request (dense all-to-all-v), freed with it
    cudaStream_t stream;
    cudaEvent_t done;
    cudaEvent_t *pending;    // event to wait on while active (own or a batch's)
    int active;
    // host-buffer starts: the request's own copy streams (upload, download), the event the
    // upload records, and the event of the last download (the next exchange waits for it)
    cudaStream_t host_up = nullptr, host_down = nullptr;
    cudaEvent_t host_up_ev = nullptr, host_down_ev = nullptr, host_mark = nullptr;
    int host_down_pending = 0;
    const char *src;         // bound buffers
    char *dst;
    int64_t src_bytes, dst_bytes;
    int64_t elem_size;
    int dtype;
    DevPool mem;             // everything the request owns
    std::vector<HostOp> ops;
    std::vector<LevelLaunch> launches;
    cudaGraphExec_t exec;
    gbx_request_info_t info;
    // maps kept for building the backward of this (forward) request
    int64_t nseg;            // standard segments (nonzero edges) in receive order
    Seg *segs_std;           // standard segments
    int32_t *srcel;          // per element: source element index in its rank's region
    int *seg_src_rank, *seg_dst_rank;
    int64_t *segv0;          // nseg + 1 segment starts (last = V)
    int64_t *send_base_copy; // P byte offsets of the send regions
    uint64_t align;          // OR of every base offset, pointer and the element size
    int64_t V;
    // locality maps
    int64_t U;
    int64_t *val_pos;        // per element (standard numbering): aggregate slot, -1 if direct
    int64_t *agg_rep_off;    // per aggregate slot: byte offset of its representative source
    int32_t *agg_dst_node;   // per aggregate slot: destination node
    int64_t Ur;              // first slot of the receive aggregate (U rounded up so that it starts
                             // 16-byte aligned: both halves of `agg` hold Ur slots)
    Seg *segs_pair;          // per node pair: aggregate block (v0 = first slot, count by next)
    int64_t npairs;
    char *agg;               // locality scratch: send aggregate | receive aggregate
    std::vector<Batch *> batches;
    // partitioned requests (kind 2): one standard-form child per non-empty send partition
    int npart = 0, nrpart = 0;
    std::vector<gbx_request_s *> parts;
    std::vector<cudaEvent_t> part_ev;
    std::vector<char> part_ready;
    int nready = 0;
    std::vector<uint32_t> feed;  // nrpart rows of ceil(npart / 32) words: send partitions feeding each
};

// Device part of a partitioned request: every forward element keyed by its send
// partition, cut into receive-contiguous runs of one source rank per partition.
struct PartPlan {
    Seg *segs = nullptr;          // all partitions' segments, partition by partition
    int32_t *idx = nullptr;       // per element, in partition order: source element in its rank's region
    std::vector<int64_t> elem_off, seg_off;   // npart + 1 each
    std::vector<uint32_t> feed;
};

// Internal steps shared by the C ABI translation unit.
int gbx_setup_forward(gbx_request_s *req, const int64_t *send_base, const int *sendcounts,
                      const int *sdispls, const int64_t *send_slot_ptr, const int *send_idx,
                      const int64_t *recv_base, const int *recvcounts, const int *rdispls,
                      const int64_t *recv_slot_ptr, const int64_t *global_sidx,
                      const int64_t *global_ridx, int want_locality);
int gbx_setup_backward(gbx_request_s *bwd, int accumulate);
int gbx_setup_partitions(gbx_request_s *parent, const gbx_request_s *f, int npart, const int64_t *part_ptr,
                         int nrpart, const int64_t *rpart_ptr, PartPlan *plan);
int gbx_setup_alltoallw(gbx_request_s *req, const int64_t *send_base, const int *sendcounts, const int64_t *sdispls,
                        const int *sendtypes, const int64_t *recv_base, const int *recvcounts, const int64_t *rdispls,
                        const int *recvtypes, const gbx_datatype_t *types, int ntypes);
int gbx_graph_setup(gbx_graph_s *g, int64_t n_in, const int *in_ptr, const int *sources,
                    int64_t n_out, const int *out_ptr, const int *dests, cudaStream_t st);
int gbx_make_copy_op(gbx_request_s *req, int level, const char *src, int src_role, char *dst,
                     int dst_role, const Seg *segs, int64_t nseg, const int32_t *idx,
                     int64_t idx_len, int64_t nelem, int64_t algo_bytes);
int gbx_validate_program(gbx_request_s *req, int64_t agg_bytes);
int gbx_split_runs(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                   int min_run, Seg **out, int64_t *out_nseg);
int gbx_make_flat_op(gbx_request_s *req, int level, const char *src, int src_role, const char *src2, int src2_role,
                     char *dst, int dst_role, const int32_t *g, int64_t nelem, int64_t dst0);
int gbx_split_single_rows(gbx_request_s *req, const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms,
                          int64_t nrows, int32_t **gs, int32_t **gd, int64_t *nsingle, int64_t **row_ptr2,
                          int64_t **row_out2, int64_t **terms2, int64_t *nmulti, int64_t *nmterms, int *ok);
int gbx_sort_pairs_by_source(gbx_request_s *req, int32_t *gs, int32_t *gd, int64_t n);
int gbx_make_flat2_op(gbx_request_s *req, int level, const char *src, int src_role, const char *src2, int src2_role,
                      char *dst, int dst_role, const int32_t *gs, const int32_t *gd, int64_t nelem);
int64_t agg_r_slot(int64_t U, int64_t s);
int gbx_make_bulk(gbx_request_s *req, const Seg *segs, int64_t nseg, int64_t nelem, bool owned, BulkTask **out, int64_t *n,
                  int *ok);
int gbx_bulk_prepare(void);
int gbx_scatter_prepare(void);
int gbx_stream_prepare(void);
int gbx_check_data_buf(const void *p, int64_t bytes);   // GBX_ERR_ARG unless the GPU can address p
// Scatter-form windows of a two-index copy whose pairs are sorted by source (gs, the source
// indices, decide the windows) and whose index arrays carry 4 elements of padding; *ok = 0
// where the form does not apply.
int gbx_make_scatter(gbx_request_s *req, const int32_t *gs, int64_t n, ScatterPiece **pieces, int64_t *npieces,
                     int *ok);
int gbx_bulk_status_take(int *status);
int gbx_make_flat(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                  int32_t **flat_idx, int64_t *dst0, int *ok);
int gbx_order_by_source(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                        int64_t src_bytes, int64_t max_piece, Seg **out, int64_t *out_nseg);
int gbx_build_fold_records(const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms, int64_t nrows,
                           longlong2 *rec, cudaStream_t st);
int gbx_make_fold_op(gbx_request_s *req, int level, char *out, int out_role, const char *bufA,
                     int a_role, const char *bufB, int b_role, const int64_t *row_ptr,
                     const int64_t *row_out, const int64_t *terms, int64_t nrows,
                     int64_t nterms, int accumulate);
