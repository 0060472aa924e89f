// gbx_move.cu -- the exchange's data-movement kernels (the hot path).
//
// gbx_copy_kernel: for every element e of a copy op, with s = elem_size,
//     dst[seg.dst_off + k*s .. +s) = src[seg.src_off + sel*s .. +s),  k = e - seg.v0,
//     sel = idx[seg.idx_off + k] (gather through the send index list) or k (contiguous)
//   This one kernel is the pack + block copy + unpack of the standard neighbourhood
//   all-to-all-v (MPI Advance section 2.2: every message, packed by its send list and
//   unpacked at its receive displacement, in one pass) and each step of the
//   locality-aware form (direct copy, gather into node-pair aggregates, one block per
//   node pair, redistribution).  Bytes are copied as opaque vectors: bit-exact.
// gbx_fold_kernel: for every row of a fold op,
//     out[row] (+)= fold over the row's groups, in order, of (fold over the group's terms)
//   with IEEE round-to-nearest adds in the payload type: the reverse exchange.
//
// Both kernels walk tiles of GBX_TILE chunks (chunk = one `vec`-byte vector) with a
// grid-stride loop; a launch may cover several ops (patterns), found by binary search
// over the tile prefix, so uneven patterns share one grid.  Consecutive threads handle
// consecutive chunks: destination writes are fully coalesced 16-byte stores, source
// reads are 16-byte vector gathers of whole elements.  No shared memory, no barriers,
// no waits: a launch always terminates.
#include "gbx_internal.cuh"

template <int VEC> struct VecT;
template <> struct VecT<16> { typedef uint4 T; };
template <> struct VecT<8> { typedef uint2 T; };
template <> struct VecT<4> { typedef unsigned int T; };
template <> struct VecT<2> { typedef unsigned short T; };
template <> struct VecT<1> { typedef unsigned char T; };

// Cache behaviour of the payload loads and stores (index and descriptor loads always go
// through L1).  GBX_LD_MODE 0: ld.global.nc; 1: + L1::no_allocate; 2: + L1::no_allocate and
// an L2 256-byte prefetch.  GBX_ST_MODE 0: st.global; 1: st.global.cs (evict first).
#ifndef GBX_LD_MODE
#define GBX_LD_MODE 0
#endif
#ifndef GBX_ST_MODE
#define GBX_ST_MODE 0
#endif

template <int VEC>
__device__ __forceinline__ typename VecT<VEC>::T ldv(const char *p) {
#if GBX_LD_MODE == 0
    return __ldg(reinterpret_cast<const typename VecT<VEC>::T *>(p));
#else
    if constexpr (VEC == 16) {
        uint4 v;
#if GBX_LD_MODE == 1
        asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
#else
        asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
            : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
#endif
        return v;
    } else {
        return __ldg(reinterpret_cast<const typename VecT<VEC>::T *>(p));
    }
#endif
}
template <int VEC>
__device__ __forceinline__ typename VecT<VEC>::T ldv_plain(const char *p) {
    return *reinterpret_cast<const typename VecT<VEC>::T *>(p);
}
template <int VEC>
__device__ __forceinline__ void stv(char *p, typename VecT<VEC>::T v) {
#if GBX_ST_MODE == 1
    if constexpr (VEC == 16) {
        __stcs(reinterpret_cast<uint4 *>(p), v);
        return;
    }
#endif
    *reinterpret_cast<typename VecT<VEC>::T *>(p) = v;
}

// Largest op index whose tile range starts at or before t.
__device__ __forceinline__ int find_op(const int64_t *__restrict__ prefix, int nops, int64_t t) {
    int lo = 0, hi = nops - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Unit (element or row) and chunk-in-unit of local chunk x of a tile whose first chunk
// is chunk r0 of unit e0.  x < GBX_TILE + cpe, so the 32-bit magic multiply is exact.
__device__ __forceinline__ uint32_t unit_of(uint32_t x, int cpe, int sh, uint32_t magic) {
    if (sh >= 0) return x >> sh;
    if (cpe < 32768) return __umulhi(x, magic);
    return x / (uint32_t)cpe;
}

// ------------------------------------------------------------------------ copy
// flat form: destinations contiguous from dst_flat0, element e reads source element
// flat_idx[e]; the index load is the only dependency of the data load
template <int VEC, int U>
__device__ __forceinline__ void copy_tile_flat(const CopyDesc *__restrict__ d, int64_t t) {
    typedef typename VecT<VEC>::T V;
    constexpr int B = GBX_TILE / U;
    const int cpe = d->cpe, sh = d->cpe_shift;
    const uint32_t magic = d->cpe_magic;
    const int64_t e0 = __ldg(d->tile_e0 + t);
    const uint32_t r0 = (uint32_t)(t * GBX_TILE - e0 * cpe);
    const int64_t left = d->nchunks - t * GBX_TILE;
    const int64_t s = d->elem_size;
    const int32_t *__restrict__ g = d->flat_idx;
    int64_t soff[U], doff[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t x = r0 + (uint32_t)(u * B) + threadIdx.x;
        const uint32_t el = unit_of(x, cpe, sh, magic);
        const int64_t j = (int64_t)(x - el * (uint32_t)cpe) * VEC;
        const int64_t e = e0 + el;
        const bool ok = (int64_t)(u * B + threadIdx.x) < left;
        const uint32_t gi = ok ? (uint32_t)__ldg(g + e) : 0u;
        // bit 31 selects the second source; offsets stay below 2^63 so the bit survives
        soff[u] = (((int64_t)(gi & ~GBX_FLAT_SRC2)) * s + j) | ((int64_t)(gi >> 31) << 62);
        doff[u] = d->dst_flat0 + e * s + j;
    }
    V val[U];
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) {
            const char *base = (soff[u] >> 62) ? d->src2 : d->src;
            val[u] = ldv<VEC>(base + (soff[u] & ((1ll << 62) - 1)));
        }
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) stv<VEC>(d->dst + doff[u], val[u]);
}

// two-index flat form: element e reads source element flat_idx[e] (bit 31 = second source)
// and writes destination element flat_didx[e]
template <int VEC, int U>
__device__ __forceinline__ void copy_tile_flat2(const CopyDesc *__restrict__ d, int64_t t) {
    typedef typename VecT<VEC>::T V;
    constexpr int B = GBX_TILE / U;
    const int cpe = d->cpe, sh = d->cpe_shift;
    const uint32_t magic = d->cpe_magic;
    const int64_t e0 = __ldg(d->tile_e0 + t);
    const uint32_t r0 = (uint32_t)(t * GBX_TILE - e0 * cpe);
    const int64_t left = d->nchunks - t * GBX_TILE;
    const int64_t s = d->elem_size;
    int64_t soff[U], doff[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t x = r0 + (uint32_t)(u * B) + threadIdx.x;
        const uint32_t el = unit_of(x, cpe, sh, magic);
        const int64_t j = (int64_t)(x - el * (uint32_t)cpe) * VEC;
        const int64_t e = e0 + el;
        const bool ok = (int64_t)(u * B + threadIdx.x) < left;
        const uint32_t gi = ok ? (uint32_t)__ldg(d->flat_idx + e) : 0u;
        const int64_t go = ok ? (int64_t)__ldg(d->flat_didx + e) : 0;
        soff[u] = (((int64_t)(gi & ~GBX_FLAT_SRC2)) * s + j) | ((int64_t)(gi >> 31) << 62);
        doff[u] = go * s + j;
    }
    V val[U];
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) {
            const char *base = (soff[u] >> 62) ? d->src2 : d->src;
            val[u] = ldv<VEC>(base + (soff[u] & ((1ll << 62) - 1)));
        }
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) stv<VEC>(d->dst + doff[u], val[u]);
}

// Software-pipelined flat forms for a single-op persistent launch: the index loads of the
// block's next tile are issued while the current tile's payload loads are in flight, so the
// payload loads no longer wait for a full index round trip.  FORM 1: flat gather, 3: two-index.
template <int VEC, int U, int FORM>
__device__ __forceinline__ void flat_indices(const CopyDesc *__restrict__ d, int64_t t, uint32_t (&gi)[U],
                                             int32_t (&gd)[U], int64_t (&e)[U], int64_t (&j)[U], bool (&ok)[U]) {
    constexpr int B = GBX_TILE / U;
    const int cpe = d->cpe, sh = d->cpe_shift;
    const uint32_t magic = d->cpe_magic;
    const int64_t e0 = __ldg(d->tile_e0 + t);
    const uint32_t r0 = (uint32_t)(t * GBX_TILE - e0 * cpe);
    const int64_t left = d->nchunks - t * GBX_TILE;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t x = r0 + (uint32_t)(u * B) + threadIdx.x;
        const uint32_t el = unit_of(x, cpe, sh, magic);
        j[u] = (int64_t)(x - el * (uint32_t)cpe) * VEC;
        e[u] = e0 + el;
        ok[u] = (int64_t)(u * B + threadIdx.x) < left;
        gi[u] = ok[u] ? (uint32_t)__ldg(d->flat_idx + e[u]) : 0u;
        if (FORM == 3) gd[u] = ok[u] ? __ldg(d->flat_didx + e[u]) : 0;
    }
}

template <int VEC, int U, int FORM>
__device__ __forceinline__ void copy_flat_pipelined(const CopyDesc *__restrict__ d, int64_t ntiles) {
    typedef typename VecT<VEC>::T V;
    const int64_t s = d->elem_size;
    int64_t t = blockIdx.x;
    if (t >= ntiles) return;
    uint32_t gi[U];
    int32_t gd[U];
    int64_t e[U], j[U];
    bool ok[U];
    flat_indices<VEC, U, FORM>(d, t, gi, gd, e, j, ok);
    for (;;) {
        const int64_t tn = t + gridDim.x;
        V val[U];
        int64_t doff[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            doff[u] = (FORM == 3 ? (int64_t)gd[u] * s : d->dst_flat0 + e[u] * s) + j[u];
            if (ok[u]) {
                const char *base = (gi[u] & GBX_FLAT_SRC2) ? d->src2 : d->src;
                val[u] = ldv<VEC>(base + (int64_t)(gi[u] & ~GBX_FLAT_SRC2) * s + j[u]);
            }
        }
        bool okc[U];
#pragma unroll
        for (int u = 0; u < U; u++) okc[u] = ok[u];
        if (tn < ntiles) flat_indices<VEC, U, FORM>(d, tn, gi, gd, e, j, ok);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (okc[u]) stv<VEC>(d->dst + doff[u], val[u]);
        if (tn >= ntiles) break;
        t = tn;
    }
}

template <int VEC, int U>
__device__ __forceinline__ void copy_tile(const CopyDesc *__restrict__ d, int64_t t) {
    typedef typename VecT<VEC>::T V;
    constexpr int B = GBX_TILE / U;
    const Seg *__restrict__ segs = d->segs;
    const int cpe = d->cpe, sh = d->cpe_shift;
    const uint32_t magic = d->cpe_magic;
    const int64_t e0 = __ldg(d->tile_e0 + t);
    const uint32_t r0 = (uint32_t)(t * GBX_TILE - e0 * cpe);
    const int64_t left = d->nchunks - t * GBX_TILE;   // chunks of this op from the tile start
    const int64_t slo = __ldg(d->tile_seg + t);
    const int64_t shi = __ldg(d->tile_seg + t + 1);

    int64_t e[U], pos[U];
    uint32_t j[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t x = r0 + (uint32_t)(u * B) + threadIdx.x;
        const uint32_t el = unit_of(x, cpe, sh, magic);
        j[u] = x - el * (uint32_t)cpe;
        e[u] = e0 + el;
        pos[u] = slo;
    }
    // branch-free search: largest segment in [slo, shi] starting at or before e[u]
    const int64_t span = shi - slo;
    int64_t step = 1;
    while (step <= span) step <<= 1;
    for (step >>= 1; step > 0; step >>= 1) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t cand = pos[u] + step;
            if (cand <= shi && __ldg(&segs[cand].v0) <= e[u]) pos[u] = cand;
        }
    }
    const int64_t s = d->elem_size;
    const int32_t *__restrict__ idx = d->idx;
#pragma unroll
    for (int u = 0; u < U; u++) {   // e[u] := source byte offset, pos[u] := destination byte offset
        const Seg *sg = segs + pos[u];
        const int64_t k = e[u] - __ldg(&sg->v0);
        const int64_t io = __ldg(&sg->idx_off);
        const bool ok = (int64_t)(u * B + threadIdx.x) < left;
        const int64_t sel = (io >= 0 && ok) ? (int64_t)__ldg(idx + io + k) : k;
        e[u] = __ldg(&sg->src_off) + sel * s + (int64_t)j[u] * VEC;
        pos[u] = __ldg(&sg->dst_off) + k * s + (int64_t)j[u] * VEC;
    }
    V val[U];
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) val[u] = ldv<VEC>(d->src + e[u]);
#pragma unroll
    for (int u = 0; u < U; u++)
        if ((int64_t)(u * B + threadIdx.x) < left) stv<VEC>(d->dst + pos[u], val[u]);
}

// VEC > 0: every op of the launch has that vector width; VEC == 0: mixed widths
// (batched patterns), dispatched per tile.  FLAT 0: segment form, 1: flat form, 3: two-index
// flat form, 2: per op.
// GBX_COPY_OCC (threads per SM the register budget must allow; 0 = no constraint) trades
// registers for resident warps.
#ifndef GBX_COPY_OCC
#define GBX_COPY_OCC 0
#endif
template <int VEC, int U>
__device__ __forceinline__ void copy_tile_any(const CopyDesc *__restrict__ d, int64_t t, int flat) {
    if ((flat & 3) == 3) copy_tile_flat2<VEC, U>(d, t);
    else if (flat) copy_tile_flat<VEC, U>(d, t);
    else copy_tile<VEC, U>(d, t);
}

template <int VEC, int U, int FLAT>
__global__ void __launch_bounds__(GBX_TILE / U, GBX_COPY_OCC ? GBX_COPY_OCC / (GBX_TILE / U) : 1)
gbx_copy_kernel(const CopyDesc *const *__restrict__ ops, const int64_t *__restrict__ prefix,
                int nops, int64_t total_tiles) {
    for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
        const CopyDesc *d = ops[op];
        const int64_t lt = t - __ldg(prefix + op);
        if (VEC) {
            if (FLAT == 1) copy_tile_flat<VEC ? VEC : 1, U>(d, lt);
            else if (FLAT == 3) copy_tile_flat2<VEC ? VEC : 1, U>(d, lt);
            else if (FLAT == 0) copy_tile<VEC ? VEC : 1, U>(d, lt);
            else copy_tile_any<VEC ? VEC : 1, U>(d, lt, d->flat);
        } else {
            const int fl = d->flat;
            switch (d->vec) {
                case 16: copy_tile_any<16, U>(d, lt, fl); break;
                case 8: copy_tile_any<8, U>(d, lt, fl); break;
                case 4: copy_tile_any<4, U>(d, lt, fl); break;
                case 2: copy_tile_any<2, U>(d, lt, fl); break;
                default: copy_tile_any<1, U>(d, lt, fl); break;
            }
        }
    }
}

// Pipelined flat forms (descriptor flat = 5: gather, 7: two-index), one op per launch,
// persistent grid; launch bounds keep two full waves of threads resident (<= 32 registers).
template <int VEC, int U, int FORM>
__global__ void __launch_bounds__(GBX_TILE / U, 2 * U)
gbx_copy_pipe_kernel(const CopyDesc *const *__restrict__ ops, const int64_t *__restrict__ prefix, int nops,
                     int64_t total_tiles) {
    (void)prefix;
    (void)nops;
    copy_flat_pipelined<VEC, U, FORM>(ops[0], total_tiles);
}

// ------------------------------------------------------------------------ bulk
// Bulk form: contiguous pieces moved through shared memory by the bulk-copy engine.  One
// thread per CTA drives a ring of GBX_BULK_STAGES buffers: a piece is loaded with
// cp.async.bulk (completion counted on the stage's mbarrier), stored back with a bulk store,
// and a stage is refilled once the store before it has read it, so several pieces per CTA
// are always in flight.  Every mbarrier wait is bounded (the main waits by the op's
// wait_limit, the drain waits by GBX_WAIT_LIMIT): a wait that gives up records status 1 for
// every op of the launch (gbx_raise), waits (bounded again) for the stage loads still in
// flight and for the stores, and leaves the kernel.
__device__ int gbx_bulk_status;

// Records a status code (1: a bounded wait gave up, 2: a piece failed its check) in the
// process-wide word and in the status word of every op of the launch: a launch that gives up
// leaves pieces of any of its ops unfinished, so each request it serves must report it.
template <typename D>
__device__ __noinline__ void gbx_raise(const D *const *__restrict__ ops, int nops, int code) {
    atomicExch(&gbx_bulk_status, code);
    for (int i = 0; i < nops; i++) {
        int *w = ops[i]->status;
        if (w) *reinterpret_cast<volatile int *>(w) = code;
    }
    __threadfence_system();
}

__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t parity, int limit = GBX_WAIT_LIMIT) {
    for (int it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(32) gbx_bulk_kernel(const CopyDesc *const *__restrict__ ops,
                                                      const int64_t *__restrict__ prefix, int nops,
                                                      int64_t ntasks) {
    extern __shared__ __align__(128) unsigned char gbx_bulk_smem[];
    __shared__ __align__(8) uint64_t bar[GBX_BULK_STAGES];
    if (threadIdx.x != 0) return;
    constexpr int S = GBX_BULK_STAGES;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(gbx_bulk_smem);
    const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(bar);
    for (int q = 0; q < S; q++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar + 8 * q) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    char *dst_of[S];
    uint32_t len_of[S], parity[S];
    bool pend[S];
#pragma unroll
    for (int q = 0; q < S; q++) {
        parity[q] = 0;
        pend[q] = false;
        dst_of[q] = nullptr;
        len_of[q] = 0;
    }
    auto load = [&](int q, int64_t t) {
        const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
        const CopyDesc *d = ops[op];
        const BulkTask k = d->bulk[t - (nops > 1 ? __ldg(prefix + op) : 0)];
        const uint32_t b = sbar + 8 * q, len = (uint32_t)k.len;
        // pieces were validated at init; a piece that is not a whole number of aligned 16-byte
        // units within one stage is recorded and skipped
        if (k.len <= 0 || k.len > GBX_BULK_BYTES || ((k.len | k.src | k.dst |
                                                      (int64_t)(uintptr_t)d->src | (int64_t)(uintptr_t)d->dst) & 15)) {
            gbx_raise(ops, nops, 2);
            dst_of[q] = nullptr;
            len_of[q] = 0;
            pend[q] = false;
            return;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(len) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(sbuf + q * GBX_BULK_BYTES), "l"(d->src + k.src), "r"(len), "r"(b)
                     : "memory");
        dst_of[q] = d->dst + k.dst;
        len_of[q] = len;
        pend[q] = true;
    };
#pragma unroll
    for (int q = 0; q < S; q++) {
        const int64_t t = blockIdx.x + (int64_t)q * gridDim.x;
        if (t < ntasks) load(q, t);
    }
    const int limit = ops[0]->wait_limit;
    bool failed = false;
    for (int64_t k = 0;; k++) {
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= ntasks) break;
        const int q = (int)(k % S);
        if (pend[q]) {
            if (!bulk_wait(sbar + 8 * q, parity[q], limit)) {
                failed = true;
                break;
            }
            parity[q] ^= 1u;
            pend[q] = false;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                         ::"l"(dst_of[q]), "r"(sbuf + q * GBX_BULK_BYTES), "r"(len_of[q])
                         : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        // refill the previous piece's stage once its store has read it
        if (k >= 1) {
            const int64_t tn = blockIdx.x + (k - 1 + S) * gridDim.x;
            if (tn < ntasks) {
                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                load((int)((k - 1) % S), tn);
            }
        }
    }
    if (failed) {
        gbx_raise(ops, nops, 1);
        for (int q = 0; q < S; q++)
            if (pend[q]) bulk_wait(sbar + 8 * q, parity[q]);
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

int gbx_bulk_prepare(void) {
    cudaError_t e = cudaFuncSetAttribute(gbx_bulk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         GBX_BULK_STAGES * GBX_BULK_BYTES);
    return e == cudaSuccess ? GBX_SUCCESS : GBX_ERR_CUDA;
}

// ----------------------------------------------------------------- scatter
// Scatter form of a two-index copy whose pairs are sorted by source: each piece is a window of
// the source.  Warp 0 is the producer: its lane 0 has the bulk-copy engine read a window's
// runs of source elements (the gaps between them are not read) and the window's source and
// destination indices into one of S shared-memory stages, completing on the stage's "full"
// mbarrier.  The other warps are consumers: they wait on "full", scatter the window's elements
// from shared memory to their destinations with 16-byte stores, and release the stage on its
// "empty" mbarrier (one arrival per consumer warp), which the producer waits on before
// refilling it.  No CTA-wide barrier is crossed after setup, so a slow warp holds back only
// its own stage.  Every wait is bounded: a consumer that gives up raises `abort`, the producer
// then stops issuing, waits (bounded) for the copies it has in flight, and every warp leaves.
template <int NT, int S>
__global__ void __launch_bounds__(NT) gbx_scatter_kernel(const CopyDesc *const *__restrict__ ops,
                                                         const int64_t *__restrict__ prefix, int nops,
                                                         int64_t npieces) {
    constexpr int NC = NT - 32;          // consumer threads
    constexpr int NCW = NC / 32;         // consumer warps: arrivals that release a stage
    extern __shared__ __align__(128) unsigned char gbx_scatter_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ ScatterPiece piece_s[S];
    __shared__ __align__(16) ScatterPiece next_s;   // the producer's next piece, fetched ahead
    __shared__ const CopyDesc *desc_s[S];
    __shared__ volatile int abort_flag;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(gbx_scatter_smem);
    const uint32_t sfull = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t sempty = (uint32_t)__cvta_generic_to_shared(empty);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; q++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sfull + 8 * q) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sempty + 8 * q), "r"(NCW) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();   // the only CTA-wide barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane != 0) return;
        // ---------------------------------------------------------------- producer
        auto fetch = [&](int64_t t, const CopyDesc *&d) {   // piece t into next_s, asynchronously
            const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
            d = ops[op];
            const char *g = reinterpret_cast<const char *>(d->scat + (t - (nops > 1 ? __ldg(prefix + op) : 0)));
            const uint32_t sl = (uint32_t)__cvta_generic_to_shared(&next_s);
#pragma unroll
            for (int i = 0; i < (int)sizeof(ScatterPiece) / 16; i++)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sl + 16 * i), "l"(g + 16 * i) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        int64_t last[S];   // last piece issued on each stage (-1: none)
#pragma unroll
        for (int q = 0; q < S; q++) last[q] = -1;
        bool stop = false;
        const CopyDesc *d = nullptr;
        const int limit = ops[0]->wait_limit;
        if (blockIdx.x < npieces) fetch(blockIdx.x, d);
        for (int64_t k = 0;; k++) {
            const int64_t t = blockIdx.x + k * gridDim.x;
            if (t >= npieces) break;
            const int q = (int)(k % S);
            if (k >= S && !bulk_wait(sempty + 8 * q, (uint32_t)((k / S - 1) & 1), limit)) {
                abort_flag = 1;
                stop = true;
                break;
            }
            if (abort_flag) {
                stop = true;
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // consumers' reads before the refill
            asm volatile("cp.async.wait_all;" ::: "memory");
            ScatterPiece P = next_s;
            const CopyDesc *pd = d;
            const int64_t tn = t + gridDim.x;
            if (tn < npieces) fetch(tn, d);   // the next piece's descriptor, while this one loads
            const int64_t i0 = (P.m0 * 4) & ~(int64_t)15, i1 = ((P.m0 + P.n) * 4 + 15) & ~(int64_t)15;
            bool good = P.len > 0 && P.len <= GBX_SCAT_WIN && P.n > 0 && P.n <= GBX_SCAT_MAXN && P.m0 >= 0 &&
                        P.nrun > 0 && P.nrun <= GBX_SCAT_RUNS &&
                        ((P.src | (int64_t)(uintptr_t)pd->src | (int64_t)(uintptr_t)pd->flat_idx |
                          (int64_t)(uintptr_t)pd->flat_didx) & 15) == 0;
            uint32_t bytes = 0;
            for (int r = 0; good && r < P.nrun; r++) {
                const uint32_t o = P.run_off[r], l = P.run_len[r];
                good = ((o | l) & 15) == 0 && l > 0 && o + l <= (uint32_t)P.len;
                bytes += l;
            }
            const uint32_t fb = sfull + 8 * q;
            if (!good) {   // validated at init; recorded, and the consumers skip it
                gbx_raise(ops, nops, 2);
                P.n = 0;
                piece_s[q] = P;
                desc_s[q] = pd;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
                continue;
            }
            piece_s[q] = P;
            desc_s[q] = pd;
            const uint32_t ilen = (uint32_t)(i1 - i0), stage = sbuf + q * GBX_SCAT_STAGE;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes + 2 * ilen)
                         : "memory");
            for (int r = 0; r < P.nrun; r++)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(stage + P.run_off[r]), "l"(pd->src + P.src + P.run_off[r]),
                             "r"((uint32_t)P.run_len[r]), "r"(fb)
                             : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(stage + GBX_SCAT_WIN), "l"(reinterpret_cast<const char *>(pd->flat_idx) + i0),
                         "r"(ilen), "r"(fb)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(stage + GBX_SCAT_WIN + GBX_SCAT_IDX),
                         "l"(reinterpret_cast<const char *>(pd->flat_didx) + i0), "r"(ilen), "r"(fb)
                         : "memory");
            last[q] = k;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (stop) {   // leave no copy in flight: wait (bounded) for the last one issued on each stage
            gbx_raise(ops, nops, 1);
            for (int q = 0; q < S; q++)
                if (last[q] >= 0) bulk_wait(sfull + 8 * q, (uint32_t)((last[q] / S) & 1));
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    const int ct = threadIdx.x - 32;
    const int limit = ops[0]->wait_limit;
    for (int64_t k = 0;; k++) {
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= npieces) break;
        const int q = (int)(k % S);
        if (!bulk_wait(sfull + 8 * q, (uint32_t)((k / S) & 1), limit)) {
            abort_flag = 1;
            break;
        }
        const CopyDesc *d = desc_s[q];
        const int64_t src0 = piece_s[q].src, m0 = piece_s[q].m0;
        const int s = (int)d->elem_size, cpe = s >> 4, len = piece_s[q].len, n = piece_s[q].n;
        const unsigned char *win = gbx_scatter_smem + q * GBX_SCAT_STAGE;
        const int32_t *ps = reinterpret_cast<const int32_t *>(win + GBX_SCAT_WIN) + (m0 & 3);
        const int32_t *pdst = reinterpret_cast<const int32_t *>(win + GBX_SCAT_WIN + GBX_SCAT_IDX) + (m0 & 3);
        char *dst = d->dst;
        for (int i = ct; i < n * cpe; i += NC) {
            const int j = i / cpe, c = i - j * cpe;
            const int64_t w = (int64_t)ps[j] * s - src0 + c * 16;
            if (w < 0 || w + 16 > len) {   // validated at init; recorded and skipped
                gbx_raise(ops, nops, 2);
                continue;
            }
            const uint4 v = *reinterpret_cast<const uint4 *>(win + w);
            stv<16>(dst + (int64_t)pdst[j] * s + c * 16, v);
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty + 8 * q) : "memory");
        if (abort_flag) break;
    }
}

// Shapes of the scatter kernel, chosen by the launch's block value: threads per CTA (one
// producer warp plus consumers), stages per CTA and CTAs per SM (each shape fills about
// 192 KB of shared memory per SM).
struct ScatShape { int nt, stages, per_sm; };
static ScatShape scatter_shape(int block) {
    if (block <= 128) return {288, 2, 4};
    if (block <= 256) return {288, 4, 2};
    if (block <= 512) return {544, 4, 2};
    return {1024, 8, 1};
}

static cudaError_t scatter_launch(int block, int grid, cudaStream_t st, const CopyDesc *const *ops,
                                  const int64_t *prefix, int nops, int64_t n) {
    const ScatShape h = scatter_shape(block);
    const size_t smem = (size_t)h.stages * GBX_SCAT_STAGE;
    if (h.stages == 2) gbx_scatter_kernel<288, 2><<<grid, 288, smem, st>>>(ops, prefix, nops, n);
    else if (h.nt == 288) gbx_scatter_kernel<288, 4><<<grid, 288, smem, st>>>(ops, prefix, nops, n);
    else if (h.nt == 544) gbx_scatter_kernel<544, 4><<<grid, 544, smem, st>>>(ops, prefix, nops, n);
    else gbx_scatter_kernel<1024, 8><<<grid, 1024, smem, st>>>(ops, prefix, nops, n);
    return cudaGetLastError();
}

int gbx_scatter_prepare(void) {
    cudaError_t e = cudaFuncSetAttribute(gbx_scatter_kernel<288, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * GBX_SCAT_STAGE);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gbx_scatter_kernel<288, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * GBX_SCAT_STAGE);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gbx_scatter_kernel<544, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * GBX_SCAT_STAGE);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gbx_scatter_kernel<1024, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 8 * GBX_SCAT_STAGE);
    return e == cudaSuccess ? GBX_SUCCESS : GBX_ERR_CUDA;
}

// ------------------------------------------------------------------ stream
// Stream form of the flat copies (FORM 1: gather into a contiguous destination run; FORM 3:
// two-index gather-scatter): the same tiles of GBX_TILE chunks, but the per-element index
// arrays, the only data whose addresses are known in advance, are streamed into a ring of S
// shared-memory stages by the bulk-copy engine, so that the payload loads never wait for an
// index load from memory.  Warp 0 is the producer: its lane 0 finds the op of the CTA's next
// tile, has the bulk-copy engine copy the tile's index range (rounded out to 16-byte
// boundaries; the index arrays carry 4 entries of padding) into a stage, completing on the
// stage's "full" mbarrier, and refills a stage once the consumers have released it on its
// "empty" mbarrier.  The other warps are consumers: per tile, each thread gathers U chunks
// (all loads issued before the stores) reading the indices from shared memory.  No CTA-wide
// barrier after setup; every wait is bounded as in the scatter kernel (a consumer that gives
// up raises `abort`, the producer stops issuing and drains its copies in flight).
#define GBX_STREAM_IDX ((GBX_TILE + 8) * 4)   // bytes of one index array per stage

template <int VEC, int FORM, int NT, int S, int U, int PS, bool ONE>
__global__ void __launch_bounds__(NT, PS) gbx_stream_kernel(const CopyDesc *const *__restrict__ ops,
                                                        const int64_t *__restrict__ prefix, int nops,
                                                        int64_t ntiles) {
    typedef typename VecT<VEC>::T V;
    constexpr int NC = NT - 32, NCW = NC / 32;
    constexpr int STAGE = GBX_STREAM_IDX * (FORM == 3 ? 2 : 1);
    extern __shared__ __align__(128) unsigned char gbx_stream_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ const CopyDesc *desc_s[S];
    __shared__ int64_t tile_s[S], efirst_s[S], ebase_s[S];
    __shared__ volatile int abort_flag;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(gbx_stream_smem);
    const uint32_t sfull = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t sempty = (uint32_t)__cvta_generic_to_shared(empty);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; q++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sfull + 8 * q) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sempty + 8 * q), "r"(NCW) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();   // the only CTA-wide barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int limit = ops[0]->wait_limit;
    if (warp == 0) {
        if (lane != 0) return;
        // ---------------------------------------------------------------- producer
        int64_t last[S];   // last tile issued on each stage (-1: none)
#pragma unroll
        for (int q = 0; q < S; q++) last[q] = -1;
        bool stop = false;
        for (int64_t k = 0;; k++) {
            const int64_t t = blockIdx.x + k * gridDim.x;
            if (t >= ntiles) break;
            const int q = (int)(k % S);
            if (k >= S && !bulk_wait(sempty + 8 * q, (uint32_t)((k / S - 1) & 1), limit)) {
                abort_flag = 1;
                stop = true;
                break;
            }
            if (abort_flag) {
                stop = true;
                break;
            }
            const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
            const CopyDesc *d = ops[op];
            const int64_t lt = t - __ldg(prefix + op);
            const int64_t cpe = d->cpe;
            const int64_t c0 = lt * GBX_TILE;
            const int64_t c1 = min(d->nchunks, c0 + GBX_TILE);
            const int64_t e_first = c0 / cpe, e_last = (c1 - 1) / cpe;
            const int64_t e_al = e_first & ~(int64_t)3, e_end = (e_last + 4) & ~(int64_t)3;
            const uint32_t bytes = (uint32_t)((e_end - e_al) * 4);
            const uint32_t fb = sfull + 8 * q, stage = sbuf + q * STAGE;
            desc_s[q] = d;
            tile_s[q] = lt;
            efirst_s[q] = e_first;
            const uintptr_t al = (uintptr_t)d->flat_idx | (FORM == 3 ? (uintptr_t)d->flat_didx : 0);
            if ((al & 15) || bytes > GBX_STREAM_IDX || c1 <= c0) {   // validated at init; recorded, skipped
                gbx_raise(ops, nops, 2);
                ebase_s[q] = -1;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
                continue;
            }
            ebase_s[q] = e_al;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // consumers' reads before the refill
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                         "r"(bytes * (FORM == 3 ? 2u : 1u))
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(stage), "l"(d->flat_idx + e_al), "r"(bytes), "r"(fb)
                         : "memory");
            if (FORM == 3)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(stage + GBX_STREAM_IDX), "l"(d->flat_didx + e_al), "r"(bytes), "r"(fb)
                             : "memory");
            last[q] = k;
        }
        if (stop) {   // leave no copy in flight: wait (bounded) for the last one issued on each stage
            gbx_raise(ops, nops, 1);
            for (int q = 0; q < S; q++)
                if (last[q] >= 0) bulk_wait(sfull + 8 * q, (uint32_t)((last[q] / S) & 1));
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    const int ct = threadIdx.x - 32;
    for (int64_t k = 0;; k++) {
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int q = (int)(k % S);
        if (!bulk_wait(sfull + 8 * q, (uint32_t)((k / S) & 1), limit)) {
            abort_flag = 1;
            break;
        }
        const int64_t e_al = ebase_s[q];
        if (ONE && e_al >= 0) {
            // ONE (every op of the launch has one chunk per element, elem_size == VEC): chunk x
            // of the tile is element e0 + x, every offset a multiple of VEC
            const CopyDesc *d = desc_s[q];
            const int64_t e0 = efirst_s[q];
            const int left = (int)min((int64_t)GBX_TILE, d->nchunks - tile_s[q] * GBX_TILE);
            const int32_t *is = reinterpret_cast<const int32_t *>(gbx_stream_smem + q * STAGE) + (e0 - e_al);
            const int32_t *ids =
                reinterpret_cast<const int32_t *>(gbx_stream_smem + q * STAGE + GBX_STREAM_IDX) + (e0 - e_al);
            const char *src = d->src, *src2 = d->src2;
            char *dst = d->dst;
            char *dtile = dst + (FORM == 3 ? 0 : d->dst_flat0 + e0 * VEC);
            for (int base = 0; base < left; base += NC * U) {
                V val[U];
                int32_t di[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int x = base + u * NC + ct;
                    if (x < left) {
                        const uint32_t gi = (uint32_t)is[x];
                        if (FORM == 3) di[u] = ids[x];
                        const char *b = (gi & GBX_FLAT_SRC2) ? src2 : src;
                        val[u] = ldv<VEC>(b + (int64_t)(gi & ~GBX_FLAT_SRC2) * VEC);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int x = base + u * NC + ct;
                    if (x < left) stv<VEC>(FORM == 3 ? dst + (int64_t)di[u] * VEC : dtile + (int64_t)x * VEC, val[u]);
                }
            }
        } else if (!ONE && e_al >= 0) {
            const CopyDesc *d = desc_s[q];
            const int cpe = d->cpe, sh = d->cpe_shift;
            const uint32_t magic = d->cpe_magic;
            const int64_t s = d->elem_size, e0 = efirst_s[q], c0 = tile_s[q] * GBX_TILE;
            const int left = (int)min((int64_t)GBX_TILE, d->nchunks - c0);
            const uint32_t r0 = (uint32_t)(c0 - e0 * cpe);   // chunk of element e0 where the tile starts
            const int32_t *is = reinterpret_cast<const int32_t *>(gbx_stream_smem + q * STAGE);
            const int32_t *ids = reinterpret_cast<const int32_t *>(gbx_stream_smem + q * STAGE + GBX_STREAM_IDX);
            const char *src = d->src, *src2 = d->src2;
            char *dst = d->dst;
            for (int base = 0; base < left; base += NC * U) {
                V val[U];
                int64_t doff[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int x = base + u * NC + ct;
                    if (x < left) {
                        const uint32_t xx = r0 + (uint32_t)x;
                        const uint32_t el = unit_of(xx, cpe, sh, magic);
                        const int64_t j = (int64_t)(xx - el * (uint32_t)cpe) * VEC;
                        const int64_t e = e0 + el;
                        const int w = (int)(e - e_al);   // < GBX_TILE + 8: inside the stage's copy
                        const uint32_t gi = (uint32_t)is[w];
                        doff[u] = (FORM == 3 ? (int64_t)ids[w] * s : d->dst_flat0 + e * s) + j;
                        const char *b = (gi & GBX_FLAT_SRC2) ? src2 : src;
                        val[u] = ldv<VEC>(b + (int64_t)(gi & ~GBX_FLAT_SRC2) * s + j);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (base + u * NC + ct < left) stv<VEC>(dst + doff[u], val[u]);
            }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty + 8 * q) : "memory");
        if (abort_flag) break;
    }
}

// Shapes of the stream kernel, chosen by the launch's block value: threads per CTA (one
// producer warp plus consumers), stages, chunks per consumer thread per pass, CTAs per SM
// (the launch bounds hold the registers to what that many CTAs need; shared memory per SM
// is at most 4 x 4 x 8,256 = 132 KB).
// Block 128 selects the narrow shape, 160 threads x 4 stages (3 for two-index copies) x 8
// CTAs per SM with 8 chunks per thread in flight: offered only where every op has one chunk
// per element (ONE) of at most 8 bytes, whose kernel fits its 48 registers; the tuner never
// gives it other ops.
struct StreamShape { int nt, stages, u, per_sm; };
static StreamShape stream_shape(int block) {
    if (block <= 128) return {160, 4, 8, 8};
    if (block <= 256) return {288, 4, 4, 4};
    return {544, 6, 2, 2};
}

template <int VEC, int FORM, bool ONE>
static cudaError_t stream_launch_v(int block, int grid, cudaStream_t st, const CopyDesc *const *ops,
                                   const int64_t *prefix, int nops, int64_t n) {
    const StreamShape h = stream_shape(block);
    constexpr int SC = FORM == 3 ? 3 : 4;   // stages of the narrow shape
    const size_t smem = (size_t)(h.nt == 160 ? SC : h.stages) * GBX_STREAM_IDX * (FORM == 3 ? 2 : 1);
    if (h.nt == 160) {
        if constexpr (ONE && VEC <= 8)
            gbx_stream_kernel<VEC, FORM, 160, SC, 8, 8, ONE><<<grid, 160, smem, st>>>(ops, prefix, nops, n);
        else
            return cudaErrorInvalidValue;   // never chosen: only one-chunk ops of vectors up to 8 bytes
    } else if (h.nt == 288)
        gbx_stream_kernel<VEC, FORM, 288, 4, 4, 4, ONE><<<grid, 288, smem, st>>>(ops, prefix, nops, n);
    else
        gbx_stream_kernel<VEC, FORM, 544, 6, 2, 2, ONE><<<grid, 544, smem, st>>>(ops, prefix, nops, n);
    return cudaGetLastError();
}

template <int VEC>
static cudaError_t stream_launch_f(int flat, int block, int grid, cudaStream_t st, const CopyDesc *const *ops,
                                   const int64_t *prefix, int nops, int64_t n) {
    switch (flat) {
        case 10: return stream_launch_v<VEC, 1, false>(block, grid, st, ops, prefix, nops, n);
        case 11: return stream_launch_v<VEC, 3, false>(block, grid, st, ops, prefix, nops, n);
        case 12: return stream_launch_v<VEC, 1, true>(block, grid, st, ops, prefix, nops, n);
        default: return stream_launch_v<VEC, 3, true>(block, grid, st, ops, prefix, nops, n);
    }
}

// flat 10 / 11: the stream forms; 12 / 13: the same when every op of the launch has one chunk
// per element (the kernel then skips the element / chunk split)
static cudaError_t stream_launch(int vec, int flat, int block, int grid, cudaStream_t st, const CopyDesc *const *ops,
                                 const int64_t *prefix, int nops, int64_t n) {
    switch (vec) {
        case 16: return stream_launch_f<16>(flat, block, grid, st, ops, prefix, nops, n);
        case 8: return stream_launch_f<8>(flat, block, grid, st, ops, prefix, nops, n);
        case 4: return stream_launch_f<4>(flat, block, grid, st, ops, prefix, nops, n);
        default: return cudaErrorInvalidValue;   // the stream form is offered for vectors of 4..16 bytes
    }
}

template <int VEC, int FORM, bool ONE>
static cudaError_t stream_attr_o() {
    cudaError_t e = cudaFuncSetAttribute(gbx_stream_kernel<VEC, FORM, 288, 4, 4, 4, ONE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         4 * GBX_STREAM_IDX * (FORM == 3 ? 2 : 1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gbx_stream_kernel<VEC, FORM, 544, 6, 2, 2, ONE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 6 * GBX_STREAM_IDX * (FORM == 3 ? 2 : 1));
    if constexpr (ONE && VEC <= 8) {
        constexpr int SC = FORM == 3 ? 3 : 4;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(gbx_stream_kernel<VEC, FORM, 160, SC, 8, 8, ONE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SC * GBX_STREAM_IDX * (FORM == 3 ? 2 : 1));
    }
    return e;
}

template <int VEC, int FORM>
static cudaError_t stream_attr_v() {
    cudaError_t e = stream_attr_o<VEC, FORM, false>();
    return e == cudaSuccess ? stream_attr_o<VEC, FORM, true>() : e;
}

int gbx_stream_prepare(void) {
    cudaError_t e = stream_attr_v<16, 1>();
    if (e == cudaSuccess) e = stream_attr_v<16, 3>();
    if (e == cudaSuccess) e = stream_attr_v<8, 1>();
    if (e == cudaSuccess) e = stream_attr_v<8, 3>();
    if (e == cudaSuccess) e = stream_attr_v<4, 1>();
    if (e == cudaSuccess) e = stream_attr_v<4, 3>();
    return e == cudaSuccess ? GBX_SUCCESS : GBX_ERR_CUDA;
}

int gbx_bulk_status_take(int *status) {
    int zero = 0;
    GBX_CUDA_TRY(cudaMemcpyFromSymbol(status, gbx_bulk_status, sizeof(int)));
    GBX_CUDA_TRY(cudaMemcpyToSymbol(gbx_bulk_status, &zero, sizeof(int)));
    return GBX_SUCCESS;
}

// ------------------------------------------------------------------------ fold
// Payload vectors: the CUDA vector type of `VEC` bytes of T, added component-wise with
// IEEE round-to-nearest adds (never contracted, never reassociated).
template <typename T, int VEC> struct PackT;
template <> struct PackT<double, 16> { typedef double2 T; };
template <> struct PackT<double, 8> { typedef double T; };
template <> struct PackT<float, 16> { typedef float4 T; };
template <> struct PackT<float, 8> { typedef float2 T; };
template <> struct PackT<float, 4> { typedef float T; };

__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
__device__ __forceinline__ double padd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float4 padd(float4 a, float4 b) {
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float padd(float a, float b) { return __fadd_rn(a, b); }

template <typename P>
__device__ __forceinline__ P pload(const char *p) { return __ldg(reinterpret_cast<const P *>(p)); }

template <typename T, int VEC, int U>
__device__ __forceinline__ void fold_tile(const FoldDesc *__restrict__ d, int64_t t) {
    typedef typename PackT<T, VEC>::T PK;
    constexpr int B = GBX_TILE / U;
    const int cpe = d->cpe, sh = d->cpe_shift;
    const uint32_t magic = d->cpe_magic;
    const int64_t e0 = __ldg(d->tile_e0 + t);
    const uint32_t r0 = (uint32_t)(t * GBX_TILE - e0 * cpe);
    const int64_t left = d->nchunks - t * GBX_TILE;
    const int64_t *__restrict__ terms = d->terms;
    // one 16-byte record per row: most rows have a single term, which it holds inline
    int64_t oa[U], ob[U];
    uint32_t jv[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t x = r0 + (uint32_t)(u * B) + threadIdx.x;
        const uint32_t el = unit_of(x, cpe, sh, magic);
        jv[u] = (x - el * (uint32_t)cpe) * VEC;
        const bool ok = (int64_t)(u * B + threadIdx.x) < left;
        if (ok) {
            const longlong2 r = __ldg(d->rec + e0 + el);
            oa[u] = r.x;
            ob[u] = r.y;
        } else {
            oa[u] = 0;
            ob[u] = 0;
        }
    }
    PK res[U];
    bool multi = false;
#pragma unroll
    for (int u = 0; u < U; u++) {
        if ((uint64_t)oa[u] & GBX_ROW_SINGLE) {
            const uint64_t w = (uint64_t)ob[u];
            res[u] = pload<PK>(((w & GBX_TERM_BUFB) ? d->bufB : d->bufA) + (int64_t)(w & GBX_TERM_MASK) + jv[u]);
        } else if ((int64_t)(u * B + threadIdx.x) < left) {
            multi = true;
        }
    }
    if (multi) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (((uint64_t)oa[u] & GBX_ROW_SINGLE) || (int64_t)(u * B + threadIdx.x) >= left) continue;
            const int64_t b = (int64_t)((uint64_t)ob[u] >> GBX_ROW_CNT_BITS);
            const int64_t n = (int64_t)((uint64_t)ob[u] & ((1ull << GBX_ROW_CNT_BITS) - 1));
            PK grp, tot;
            bool has = false;
            for (int64_t m = 0; m < n; m++) {
                const uint64_t w = (uint64_t)__ldg(terms + b + m);
                const PK x = pload<PK>(((w & GBX_TERM_BUFB) ? d->bufB : d->bufA) + (int64_t)(w & GBX_TERM_MASK) + jv[u]);
                if (m == 0) {
                    grp = x;
                } else if (w & GBX_TERM_GROUP) {
                    tot = has ? padd(tot, grp) : grp;
                    has = true;
                    grp = x;
                } else {
                    grp = padd(grp, x);
                }
            }
            res[u] = has ? padd(tot, grp) : grp;
        }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        if ((int64_t)(u * B + threadIdx.x) >= left) continue;
        PK *o = reinterpret_cast<PK *>(d->out + (oa[u] & (int64_t)~GBX_ROW_SINGLE) + jv[u]);
        PK r = res[u];
        if (d->accumulate) r = padd(*o, r);
        *o = r;
    }
}

// Stream form of the fold (the reverse exchange's sums): the fold's tiles, with each tile's
// row records and its rows' term lists (both contiguous ranges, the terms rounded out to
// 16-byte boundaries; the term arrays carry 2 entries of padding) copied into a ring of S
// shared-memory stages by the bulk-copy engine from one producer lane, completing on the
// stage's "full" mbarrier.  Each consumer thread then holds one chunk of one row: it reads
// the record and terms from shared memory and issues up to GBX_SFOLD_K gradient loads of
// the row at once before adding them in the row's fixed order, so a row costs one memory
// latency instead of two per term.  A tile whose terms do not fit a stage reads them from
// global memory.  Waits bounded as in the stream copy.
#define GBX_SFOLD_REC ((GBX_TILE + 2) * 16)   // bytes of records per stage
#define GBX_SFOLD_TERMS 2048                   // term entries per stage
#define GBX_SFOLD_STAGE (GBX_SFOLD_REC + GBX_SFOLD_TERMS * 8)
// gradient loads in flight per thread: 8 of 4 or 8 bytes, 4 of 16 bytes (the registers of
// 2 CTAs of 544 threads per SM)

template <typename T, int VEC, int NT, int S, int PS>
__global__ void __launch_bounds__(NT, PS) gbx_sfold_kernel(const FoldDesc *const *__restrict__ ops,
                                                           const int64_t *__restrict__ prefix, int nops,
                                                           int64_t ntiles) {
    typedef typename PackT<T, VEC>::T PK;
    constexpr int NC = NT - 32, NCW = NC / 32;
    constexpr int GBX_SFOLD_K = VEC == 16 ? 4 : 8;
    extern __shared__ __align__(128) unsigned char gbx_sfold_smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ const FoldDesc *desc_s[S];
    __shared__ int64_t tile_s[S], rfirst_s[S], tbase_s[S];
    __shared__ volatile int abort_flag;
    const uint32_t sbuf = (uint32_t)__cvta_generic_to_shared(gbx_sfold_smem);
    const uint32_t sfull = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t sempty = (uint32_t)__cvta_generic_to_shared(empty);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; q++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sfull + 8 * q) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sempty + 8 * q), "r"(NCW) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();   // the only CTA-wide barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int limit = ops[0]->wait_limit;
    if (warp == 0) {
        if (lane != 0) return;
        // ---------------------------------------------------------------- producer
        int64_t last[S];
#pragma unroll
        for (int q = 0; q < S; q++) last[q] = -1;
        bool stop = false;
        for (int64_t k = 0;; k++) {
            const int64_t t = blockIdx.x + k * gridDim.x;
            if (t >= ntiles) break;
            const int q = (int)(k % S);
            if (k >= S && !bulk_wait(sempty + 8 * q, (uint32_t)((k / S - 1) & 1), limit)) {
                abort_flag = 1;
                stop = true;
                break;
            }
            if (abort_flag) {
                stop = true;
                break;
            }
            const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
            const FoldDesc *d = ops[op];
            const int64_t lt = t - __ldg(prefix + op);
            const int64_t cpe = d->cpe, c0 = lt * GBX_TILE, c1 = min(d->nchunks, c0 + GBX_TILE);
            const int64_t r_first = c0 / cpe, r_last = (c1 - 1) / cpe;
            const uint32_t rbytes = (uint32_t)((r_last - r_first + 1) * 16);
            const int64_t tb = __ldg(d->row_ptr + r_first), te = __ldg(d->row_ptr + r_last + 1);
            const int64_t tb_al = tb & ~(int64_t)1, te_al = (te + 1) & ~(int64_t)1;
            const bool inl = (te_al - tb_al) <= GBX_SFOLD_TERMS;
            const uint32_t tbytes = inl ? (uint32_t)((te_al - tb_al) * 8) : 0u;
            const uint32_t fb = sfull + 8 * q, stage = sbuf + q * GBX_SFOLD_STAGE;
            desc_s[q] = d;
            tile_s[q] = lt;
            rfirst_s[q] = r_first;
            tbase_s[q] = inl ? tb_al : -1;
            const uintptr_t al = (uintptr_t)d->rec | (uintptr_t)d->terms;
            if ((al & 15) || rbytes > GBX_SFOLD_REC || c1 <= c0) {   // validated at init; recorded, skipped
                gbx_raise(ops, nops, 2);
                rfirst_s[q] = -1;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fb) : "memory");
                continue;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(rbytes + tbytes)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(stage), "l"(d->rec + r_first), "r"(rbytes), "r"(fb)
                         : "memory");
            if (tbytes)
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             ::"r"(stage + GBX_SFOLD_REC), "l"(d->terms + tb_al), "r"(tbytes), "r"(fb)
                             : "memory");
            last[q] = k;
        }
        if (stop) {
            gbx_raise(ops, nops, 1);
            for (int q = 0; q < S; q++)
                if (last[q] >= 0) bulk_wait(sfull + 8 * q, (uint32_t)((last[q] / S) & 1));
        }
        return;
    }
    // -------------------------------------------------------------------- consumers
    const int ct = threadIdx.x - 32;
    for (int64_t k = 0;; k++) {
        const int64_t t = blockIdx.x + k * gridDim.x;
        if (t >= ntiles) break;
        const int q = (int)(k % S);
        if (!bulk_wait(sfull + 8 * q, (uint32_t)((k / S) & 1), limit)) {
            abort_flag = 1;
            break;
        }
        const int64_t r_first = rfirst_s[q];
        if (r_first >= 0) {
            const FoldDesc *d = desc_s[q];
            const int cpe = d->cpe, sh = d->cpe_shift;
            const uint32_t magic = d->cpe_magic;
            const int64_t c0 = tile_s[q] * GBX_TILE, tb_al = tbase_s[q];
            const int left = (int)min((int64_t)GBX_TILE, d->nchunks - c0);
            const uint32_t r0 = (uint32_t)(c0 - r_first * cpe);
            const longlong2 *rs = reinterpret_cast<const longlong2 *>(gbx_sfold_smem + q * GBX_SFOLD_STAGE);
            const int64_t *ts = reinterpret_cast<const int64_t *>(gbx_sfold_smem + q * GBX_SFOLD_STAGE + GBX_SFOLD_REC);
            const char *bufA = d->bufA, *bufB = d->bufB;
            for (int x = ct; x < left; x += NC) {
                const uint32_t xx = r0 + (uint32_t)x;
                const uint32_t el = unit_of(xx, cpe, sh, magic);
                const int64_t jv = (int64_t)(xx - el * (uint32_t)cpe) * VEC;
                const longlong2 rec = rs[el];
                const uint64_t oa = (uint64_t)rec.x, ob = (uint64_t)rec.y;
                PK res;
                if (oa & GBX_ROW_SINGLE) {
                    res = pload<PK>(((ob & GBX_TERM_BUFB) ? bufB : bufA) + (int64_t)(ob & GBX_TERM_MASK) + jv);
                } else {
                    const int64_t b = (int64_t)(ob >> GBX_ROW_CNT_BITS);
                    const int n = (int)(ob & ((1ull << GBX_ROW_CNT_BITS) - 1));
                    const int64_t *tw = tb_al >= 0 ? ts + (b - tb_al) : d->terms + b;
                    PK grp, tot;
                    bool has = false;
                    for (int m0 = 0; m0 < n; m0 += GBX_SFOLD_K) {
                        const int cnt = min(GBX_SFOLD_K, n - m0);
                        PK xv[GBX_SFOLD_K];
                        uint32_t gbit = 0;
#pragma unroll
                        for (int i = 0; i < GBX_SFOLD_K; i++)
                            if (i < cnt) {
                                const uint64_t w = (uint64_t)tw[m0 + i];
                                gbit |= (w & GBX_TERM_GROUP) ? (1u << i) : 0u;
                                xv[i] = pload<PK>(((w & GBX_TERM_BUFB) ? bufB : bufA) + (int64_t)(w & GBX_TERM_MASK) + jv);
                            }
#pragma unroll
                        for (int i = 0; i < GBX_SFOLD_K; i++)
                            if (i < cnt) {
                                if (m0 + i == 0) {
                                    grp = xv[i];
                                } else if (gbit & (1u << i)) {
                                    tot = has ? padd(tot, grp) : grp;
                                    has = true;
                                    grp = xv[i];
                                } else {
                                    grp = padd(grp, xv[i]);
                                }
                            }
                    }
                    res = has ? padd(tot, grp) : grp;
                }
                PK *o = reinterpret_cast<PK *>(d->out + (int64_t)(oa & ~GBX_ROW_SINGLE) + jv);
                if (d->accumulate) res = padd(*o, res);
                *o = res;
            }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sempty + 8 * q) : "memory");
        if (abort_flag) break;
    }
}

#define GBX_SFOLD_NT 544
#define GBX_SFOLD_S 3

template <typename T, int VEC>
static cudaError_t sfold_launch_v(int grid, cudaStream_t st, const FoldDesc *const *ops, const int64_t *prefix,
                                  int nops, int64_t n) {
    gbx_sfold_kernel<T, VEC, GBX_SFOLD_NT, GBX_SFOLD_S, 2>
        <<<grid, GBX_SFOLD_NT, GBX_SFOLD_S * GBX_SFOLD_STAGE, st>>>(ops, prefix, nops, n);
    return cudaGetLastError();
}

template <typename T, int VEC>
static cudaError_t sfold_attr_v() {
    return cudaFuncSetAttribute(gbx_sfold_kernel<T, VEC, GBX_SFOLD_NT, GBX_SFOLD_S, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, GBX_SFOLD_S * GBX_SFOLD_STAGE);
}

int gbx_sfold_prepare(void) {
    cudaError_t e = sfold_attr_v<double, 16>();
    if (e == cudaSuccess) e = sfold_attr_v<double, 8>();
    if (e == cudaSuccess) e = sfold_attr_v<float, 16>();
    if (e == cudaSuccess) e = sfold_attr_v<float, 8>();
    if (e == cudaSuccess) e = sfold_attr_v<float, 4>();
    return e == cudaSuccess ? GBX_SUCCESS : GBX_ERR_CUDA;
}

// CLS 1..5: every op of the launch is (f64,16) (f64,8) (f32,16) (f32,8) (f32,4);
// CLS 0: mixed (batched patterns), dispatched per tile.  The single-payload kernels with one
// chunk per thread (1024-thread blocks) are held to 32 registers so that two blocks fit on
// an SM: the fold is bound by load latency, and the doubled occupancy outweighs the few
// bytes of spill this costs (512^3 backward, all rows folded: 0.90 -> 0.82 ms).
template <int CLS, int U>
__global__ void __launch_bounds__(GBX_TILE / U, (U == 1 && CLS != 0) ? 2 : 1)
gbx_fold_kernel(const FoldDesc *const *__restrict__ ops, const int64_t *__restrict__ prefix,
                int nops, int64_t total_tiles) {
    for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        const int op = nops > 1 ? find_op(prefix, nops, t) : 0;
        const FoldDesc *d = ops[op];
        const int64_t lt = t - __ldg(prefix + op);
        const int cls = CLS ? CLS : (d->dtype == GBX_F64 ? (d->vec == 16 ? 1 : 2)
                                                         : (d->vec == 16 ? 3 : d->vec == 8 ? 4 : 5));
        switch (cls) {
            case 1: fold_tile<double, 16, U>(d, lt); break;
            case 2: fold_tile<double, 8, U>(d, lt); break;
            case 3: fold_tile<float, 16, U>(d, lt); break;
            case 4: fold_tile<float, 8, U>(d, lt); break;
            default: fold_tile<float, 4, U>(d, lt); break;
        }
    }
}

// ------------------------------------------------------------------- launching
static int g_num_sms = 0;

int gbx_num_sms(void) {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

typedef void (*CopyFn)(const CopyDesc *const *, const int64_t *, int, int64_t);
typedef void (*FoldFn)(const FoldDesc *const *, const int64_t *, int, int64_t);

template <int VEC, int FLAT>
static CopyFn copy_fn_u(int block) {
    switch (block) {
        case 128: return gbx_copy_kernel<VEC, 8, FLAT>;
        case 256: return gbx_copy_kernel<VEC, 4, FLAT>;
        case 512: return gbx_copy_kernel<VEC, 2, FLAT>;
        default: return gbx_copy_kernel<VEC, 1, FLAT>;
    }
}

template <int VEC, int FORM>
static CopyFn pipe_fn_u(int block) {
    return block == 1024 ? gbx_copy_pipe_kernel<VEC, 1, FORM> : gbx_copy_pipe_kernel<VEC, 2, FORM>;
}

template <int VEC>
static CopyFn copy_fn_v(int block, int flat) {
    if (flat == 5) return pipe_fn_u<VEC, 1>(block);
    if (flat == 7) return pipe_fn_u<VEC, 3>(block);
    if (flat == 1) return copy_fn_u<VEC, 1>(block);
    if (flat == 3) return copy_fn_u<VEC, 3>(block);
    if (flat == 0) return copy_fn_u<VEC, 0>(block);
    return copy_fn_u<VEC, 2>(block);
}

// flat: 0 segment form, 1 flat form, 3 two-index flat form, 2 decided per op (mixed launches),
// 5 / 7 the pipelined flat forms (one op, persistent grid, block 512 or 1024)
static CopyFn copy_fn(int vec, int block, int flat) {
    switch (vec) {
        case 16: return copy_fn_v<16>(block, flat);
        case 8: return copy_fn_v<8>(block, flat);
        case 4: return copy_fn_v<4>(block, flat);
        case 2: return copy_fn_v<2>(block, flat);
        case 1: return copy_fn_v<1>(block, flat);
        default:   // mixed widths: U <= 4
            switch (block) {
                case 512: return gbx_copy_kernel<0, 2, 2>;
                case 1024: return gbx_copy_kernel<0, 1, 2>;
                default: return gbx_copy_kernel<0, 4, 2>;
            }
    }
}

template <int CLS>
static FoldFn fold_fn_u(int block) {
    switch (block) {
        case 128: return gbx_fold_kernel<CLS, 8>;
        case 256: return gbx_fold_kernel<CLS, 4>;
        case 512: return gbx_fold_kernel<CLS, 2>;
        default: return gbx_fold_kernel<CLS, 1>;
    }
}

static int fold_cls(int dtype, int vec) {
    if (vec == 0) return 0;
    if (dtype == GBX_F64) return vec == 16 ? 1 : 2;
    return vec == 16 ? 3 : vec == 8 ? 4 : 5;
}

static FoldFn fold_fn(int dtype, int vec, int block) {
    switch (fold_cls(dtype, vec)) {
        case 1: return fold_fn_u<1>(block);
        case 2: return fold_fn_u<2>(block);
        case 3: return fold_fn_u<3>(block);
        case 4: return fold_fn_u<4>(block);
        case 5: return fold_fn_u<5>(block);
        default: return block == 128 ? gbx_fold_kernel<0, 4> : fold_fn_u<0>(block);
    }
}

// Blocks of the mixed kernels never go below 256 threads (their unroll is capped at 4).
int gbx_effective_block(int vec_class, int block) { return (vec_class == 0 && block < 256) ? 256 : block; }

static int pipe_block(int flat, int block) { return (flat == 5 || flat == 7) && block < 512 ? 512 : block; }

int gbx_occupancy(int kind, int dtype, int vec, int block, int flat) {
    if (kind == 1 && flat == 1) return 2;   // stream fold: two CTAs of 544 threads per SM
    if (kind == 0 && flat == 8) return 1;   // bulk kernel: one CTA per SM (its ring)
    if (kind == 0 && flat == 9) return scatter_shape(block).per_sm;
    if (kind == 0 && flat >= 10 && flat <= 13) return stream_shape(block).per_sm;
    if (kind == 0) block = pipe_block(flat, block);
    const void *f = kind == 0 ? (const void *)copy_fn(vec, block, flat) : (const void *)fold_fn(dtype, vec, block);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, gbx_effective_block(vec, block), 0);
    return n > 0 ? n : 1;
}

static int clamp_grid(int grid, int64_t total_tiles) {
    if (grid <= 0 || grid > total_tiles) grid = (int)(total_tiles < (1ll << 30) ? total_tiles : (1ll << 30));
    return grid;
}

cudaError_t gbx_launch_copy(const CopyDesc *const *ops, const int64_t *tile_prefix, int nops, int64_t total_tiles,
                            int vec, int flat, int block, int grid, cudaStream_t st) {
    if (total_tiles <= 0) return cudaSuccess;
    if (flat == 8) {   // bulk form: a "tile" is one piece
        gbx_bulk_kernel<<<clamp_grid(grid, total_tiles), 32, GBX_BULK_STAGES * GBX_BULK_BYTES, st>>>(
            ops, tile_prefix, nops, total_tiles);
        return cudaGetLastError();
    }
    if (flat == 9) {   // scatter form: a "tile" is one source window
        return scatter_launch(block, clamp_grid(grid, total_tiles), st, ops, tile_prefix, nops, total_tiles);
    }
    if (flat >= 10 && flat <= 13) {   // stream forms: the flat forms' tiles, indices through shared memory
        if (block <= 128 && !(flat >= 12 && vec <= 8)) block = 256;   // the narrow shape needs ONE, vec <= 8
        return stream_launch(vec, flat, block, clamp_grid(grid, total_tiles), st, ops, tile_prefix, nops, total_tiles);
    }
    if ((flat == 5 || flat == 7) && (nops > 1 || vec == 0)) flat -= 4;   // the pipelined kernels take one op
    block = pipe_block(flat, block);
    CopyFn f = copy_fn(vec, block, flat);
    f<<<clamp_grid(grid, total_tiles), gbx_effective_block(vec, block), 0, st>>>(ops, tile_prefix, nops, total_tiles);
    return cudaGetLastError();
}

cudaError_t gbx_launch_fold(const FoldDesc *const *ops, const int64_t *tile_prefix, int nops, int64_t total_tiles,
                            int dtype, int vec, int block, int grid, cudaStream_t st, int form) {
    if (total_tiles <= 0) return cudaSuccess;
    if (form == 1 && vec != 0) {   // stream form: one payload class per launch
        const int g = clamp_grid(grid, total_tiles);
        switch (fold_cls(dtype, vec)) {
            case 1: return sfold_launch_v<double, 16>(g, st, ops, tile_prefix, nops, total_tiles);
            case 2: return sfold_launch_v<double, 8>(g, st, ops, tile_prefix, nops, total_tiles);
            case 3: return sfold_launch_v<float, 16>(g, st, ops, tile_prefix, nops, total_tiles);
            case 4: return sfold_launch_v<float, 8>(g, st, ops, tile_prefix, nops, total_tiles);
            case 5: return sfold_launch_v<float, 4>(g, st, ops, tile_prefix, nops, total_tiles);
            default: return cudaErrorInvalidValue;
        }
    }
    FoldFn f = fold_fn(dtype, vec, block);
    f<<<clamp_grid(grid, total_tiles), gbx_effective_block(vec, block), 0, st>>>(ops, tile_prefix, nops, total_tiles);
    return cudaGetLastError();
}

// tile_e0[t] = first unit of tile t; tile_seg[t] = segment holding it (copy ops);
// tile_seg[ntiles] = nseg - 1
__global__ void tile_meta_kernel(const Seg *__restrict__ segs, int64_t nseg, int cpe, int64_t ntiles,
                                 int64_t *ts, int64_t *te0) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t == ntiles) {
            if (ts) ts[t] = nseg - 1;
            continue;
        }
        const int64_t e = (t * GBX_TILE) / cpe;
        te0[t] = e;
        if (!ts) continue;
        int64_t lo = 0, hi = nseg - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (segs[mid].v0 <= e) lo = mid; else hi = mid - 1;
        }
        ts[t] = lo;
    }
}

int gbx_build_tile_meta(const Seg *segs, int64_t nseg, int cpe, int64_t ntiles, int64_t *tile_seg,
                        int64_t *tile_e0, cudaStream_t st) {
    int64_t n = ntiles + 1;
    int64_t g = ceil_div(n, 256);
    if (g > 65535 * 16) g = 65535 * 16;
    tile_meta_kernel<<<(unsigned)g, 256, 0, st>>>(segs, nseg, cpe, ntiles, tile_seg, tile_e0);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_SUCCESS;
}
