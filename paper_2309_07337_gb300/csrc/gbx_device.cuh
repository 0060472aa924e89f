// gbx_device.cuh -- the device-side data model of the move kernels: tile size, the copy
// and fold descriptors, segment and fold-record layouts.  Everything a move kernel reads
// is defined here or in gbx_move.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#define GBX_TILE 1024                    // chunks per tile (block * unroll)
#define GBX_TERM_GROUP (1ull << 63)      // fold term: first term of a group
#define GBX_TERM_BUFB (1ull << 62)       // fold term: reads buffer B (else A)
#define GBX_TERM_MASK ((1ull << 62) - 1)
// fold row record: a = output byte offset | GBX_ROW_SINGLE; b = the row's only term when
// GBX_ROW_SINGLE is set, else (first term index << 24) | term count
#define GBX_ROW_SINGLE (1ull << 63)
#define GBX_ROW_CNT_BITS 24

#define GBX_ERR_NONE 0x7fffffff          // device error word: "no error yet"

// Buffer roles of an op's pointers (for re-binding).
enum { ROLE_SRC = 0, ROLE_DST = 1, ROLE_AGG = 2, ROLE_NONE = 3 };

struct Seg {
    int64_t v0;       // first element of the segment in the op's element space
    int64_t dst_off;  // byte offset of the segment's first destination element
    int64_t src_off;  // byte offset of the source base (contiguous: of the first element)
    int64_t idx_off;  // >= 0: element k reads index idx[idx_off + k]; < 0: contiguous
};

struct CopyDesc {
    const char *src;
    char *dst;
    const Seg *segs;
    const int32_t *idx;
    const int64_t *tile_seg;  // ntiles + 1: segment holding each tile's first element
    const int64_t *tile_e0;   // ntiles: first element of each tile
    int64_t nseg, nelem, nchunks, ntiles, elem_size;
    int32_t vec, cpe, cpe_shift;  // chunks per element; log2 of it, or -1
    uint32_t cpe_magic;           // ceil(2^32 / cpe) when cpe is not a power of two
    int32_t src_role, dst_role;
    // flat form (when set): destinations are one contiguous run from dst_flat0 and element
    // e reads source element flat_idx[e]; no segment search
    int32_t flat;
    const int32_t *flat_idx;
    int64_t dst_flat0;
    // flat form with two sources: an index with bit 31 set reads src2 (e.g. the receive
    // aggregate) instead of src
    const char *src2;
    int32_t src2_role;
    // two-index flat form (flat == 3): element e also writes destination element flat_didx[e]
    const int32_t *flat_didx;
    // bulk form (flat == 8): contiguous pieces moved by the bulk-copy engine
    const struct BulkTask *bulk;
    int64_t nbulk;
    // scatter form (flat == 9) of a two-index copy whose pairs (flat_idx, flat_didx) are sorted
    // by source: the sources are read a window at a time by the bulk-copy engine and
    // scattered from shared memory by the threads
    const struct ScatterPiece *scat;
    int64_t nscat;
    // the waiting kernels (bulk, scatter): the request's status word (host-mapped memory,
    // read by gbx_wait / gbx_test), set to 1 when a bounded wait gave up and 2 when a piece
    // failed its in-kernel check; and the spin limit of their main waits (the waits that
    // drain copies already in flight keep GBX_WAIT_LIMIT)
    int *status;
    int32_t wait_limit;
};
#define GBX_WAIT_LIMIT (1 << 22)

// One window of a scatter-form copy: the source elements of sorted pairs m0 .. m0+n-1 lie in
// nrun runs of contiguous source bytes, run r at [src + run_off[r], src + run_off[r] +
// run_len[r]) (16-byte multiples, ascending, disjoint, inside [src, src + len), len at most
// GBX_SCAT_WIN); the gaps between runs hold no pair's source and are not read.
#define GBX_SCAT_RUNS 24
#define GBX_SCAT_GAP 1024   // gaps up to this many bytes are read with their run
struct ScatterPiece {
    int64_t src, m0;
    int32_t len, n, nrun, pad;
    uint16_t run_off[GBX_SCAT_RUNS], run_len[GBX_SCAT_RUNS];
};

// One piece of a bulk-form copy: len bytes (a multiple of 16, at most GBX_BULK_BYTES) from
// byte src of the op's source to byte dst of its destination, both 16-byte aligned.
struct BulkTask {
    int64_t src, dst, len;
};
#define GBX_BULK_BYTES 32768             // bytes per bulk piece (one shared-memory stage)
#define GBX_BULK_STAGES 4                // stages per CTA of the bulk kernel
// scatter form: a stage holds one source window of GBX_SCAT_WIN bytes, then the window's
// source indices and its destination indices (at most GBX_SCAT_MAXN pairs, each index copy
// rounded out to 16-byte boundaries, so the index arrays carry 4 elements of padding)
#define GBX_SCAT_WIN 16384
#define GBX_SCAT_MAXN (GBX_SCAT_WIN / 16)
#define GBX_SCAT_IDX (GBX_SCAT_MAXN * 4 + 16)
#define GBX_SCAT_STAGE (GBX_SCAT_WIN + 2 * GBX_SCAT_IDX)
#define GBX_FLAT_SRC2 0x80000000u

struct FoldDesc {
    char *out;
    const char *bufA;
    const char *bufB;
    const int64_t *row_ptr;   // nrows + 1 (setup and validation)
    const int64_t *row_out;   // byte offset of each row's output element (setup and validation)
    const longlong2 *rec;     // nrows packed row records (the kernel's view)
    const int64_t *terms;     // byte offset | GBX_TERM_GROUP | GBX_TERM_BUFB
    const int64_t *tile_e0;   // ntiles: first row of each tile
    int64_t nrows, nchunks, ntiles, elem_size;
    int32_t vec, cpe, cpe_shift;
    uint32_t cpe_magic;
    int32_t dtype, accumulate;
    int32_t out_role, a_role, b_role;
    int *status;              // the request's status word (see CopyDesc)
    int32_t wait_limit;
};
