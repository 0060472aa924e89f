// gbx_alltoallw.cu -- device-side setup of the persistent neighbourhood all-to-all-w.
//
// MPI_Neighbor_alltoallw (the neighbourhood collectives of MPI Advance, section 2.2, with
// one datatype per edge; the MPI standard's meaning) is lowered, once at init, onto the
// standard exchange's move program:
//   1. per matched edge: datatype index, count, displacement and bound checks, and the
//      message length in bytes (the two sides must agree);
//   2. the unit u: the largest power of two <= 16 dividing every offset and length, so
//      that every message is a sequence of whole u-byte units on both sides;
//   3. per unit: its send and receive byte addresses, walking both type maps;
//   4. a sort of the receive addresses (a repeated address is a receive byte written
//      twice), then a sort into (destination rank, receive address) order;
//   5. receive-contiguous runs of one source rank become segments, the units' source
//      offsets their index list -- the same form as the all-to-all-v with a send index
//      list, so the copy kernels, the autotuner and the reverse exchange apply unchanged.
// Errors go to a device word with atomicMin (lowest code wins); nothing moves on error.
#include <algorithm>
#include <cstring>

#include "gbx_internal.cuh"

#define WT 256
#define W_EACH(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static unsigned wgrid(int64_t n) {
    int64_t g = ceil_div(n > 0 ? n : 1, WT);
    return (unsigned)(g > 65535ll * 32 ? 65535ll * 32 : g);
}

namespace {

constexpr int64_t kTypeMaxSize = 1ll << 31;
constexpr int64_t kAddrLimit = 1ll << 62;

struct WArgs {
    const int *out_owner, *in_owner;
    const int64_t *match_in;
    const int *sendcounts, *sendtypes, *recvcounts, *recvtypes;
    const int64_t *sdispls, *rdispls, *send_base, *recv_base;
    const gbx_datatype_t *types;
    int ntypes, P;
    int64_t E, send_bytes, recv_bytes;
};

__device__ __forceinline__ void wset_err(int *err, int code) { atomicMin(err, code); }

__device__ __forceinline__ int64_t wtype_size(const gbx_datatype_t &t) {
    return t.blocklen * t.count[0] * t.count[1] * t.count[2];
}

// One past the last byte of `cnt` items (cnt > 0, size > 0), or kAddrLimit when that
// exceeds 2^62 (any such span lies outside every buffer).
__device__ int64_t wspan(const gbx_datatype_t &t, int64_t cnt) {
    int64_t s = t.blocklen;
    const int64_t terms[4][2] = {{cnt - 1, t.extent}, {t.count[0] - 1, t.stride[0]},
                                 {t.count[1] - 1, t.stride[1]}, {t.count[2] - 1, t.stride[2]}};
    for (int l = 0; l < 4; l++) {
        const int64_t n = terms[l][0], st = terms[l][1];
        if (n > 0 && st > 0) {
            if (n > (kAddrLimit - s) / st) return kAddrLimit;
            s += n * st;
        }
    }
    return s;
}

// Offset (from the message's displacement) of byte b of the type-map sequence.
__device__ __forceinline__ int64_t wtype_byte(const gbx_datatype_t &t, int64_t b) {
    const int64_t size = wtype_size(t);
    const int64_t item = b / size, w = b - item * size;
    int64_t blk = w / t.blocklen;
    const int64_t off = w - blk * t.blocklen;
    const int64_t c0 = blk % t.count[0];
    blk /= t.count[0];
    const int64_t c1 = blk % t.count[1];
    const int64_t c2 = blk / t.count[1];
    return item * t.extent + c2 * t.stride[2] + c1 * t.stride[1] + c0 * t.stride[0] + off;
}

__global__ void w_base_kernel(WArgs a, int *err, unsigned long long *align) {
    W_EACH(r, (int64_t)a.P) {
        if (a.send_base[r] < 0 || a.recv_base[r] < 0) wset_err(err, GBX_ERR_INDEX);
        atomicOr(align, (unsigned long long)a.send_base[r] | (unsigned long long)a.recv_base[r]);
    }
}

// per in-edge i: checks, and the message length in bytes (0 when the edge is in error)
__global__ void w_edge_kernel(WArgs a, int64_t *nbytes, int *err, unsigned long long *align) {
    W_EACH(i, a.E) {
        nbytes[i] = 0;
        const int64_t e = a.match_in[i];
        const int r = a.out_owner[e], d = a.in_owner[i];
        const int ts = a.sendtypes[e], tr = a.recvtypes[i];
        if (ts < 0 || ts >= a.ntypes || tr < 0 || tr >= a.ntypes) { wset_err(err, GBX_ERR_ARG); continue; }
        const gbx_datatype_t Ts = a.types[ts], Tr = a.types[tr];
        const int64_t sc = a.sendcounts[e], rc = a.recvcounts[i];
        const int64_t n = sc * wtype_size(Ts);
        if (sc < 0 || rc < 0 || n != rc * wtype_size(Tr)) { wset_err(err, GBX_ERR_TRUNCATE); continue; }
        const int64_t sd = a.sdispls[e], rd = a.rdispls[i];
        if (sd < 0 || rd < 0) { wset_err(err, GBX_ERR_INDEX); continue; }
        if (a.send_base[r] < 0 || a.recv_base[d] < 0) continue;   // reported by w_base_kernel
        atomicOr(align, (unsigned long long)sd | (unsigned long long)rd);
        if (n == 0) continue;
        const int64_t sh = wspan(Ts, sc), rh = wspan(Tr, rc);
        // every term below stays within +-2^63: bases and displacements are first bounded
        if (a.send_base[r] > a.send_bytes || sd > a.send_bytes || a.recv_base[d] > a.recv_bytes ||
            rd > a.recv_bytes || sh > a.send_bytes - a.send_base[r] - sd || rh > a.recv_bytes - a.recv_base[d] - rd) {
            wset_err(err, GBX_ERR_INDEX);
            continue;
        }
        nbytes[i] = n;
    }
}

__global__ void w_units_kernel(const int64_t *nbytes, int64_t E, int64_t u, int64_t *nunits, int64_t *nonzero) {
    W_EACH(i, E) {
        nunits[i] = nbytes[i] / u;
        nonzero[i] = nbytes[i] > 0;
    }
}

// per unit x (in-edge order): send / receive byte addresses, ranks, overlap key
__global__ void w_expand_kernel(WArgs a, const int64_t *uoff, int64_t N, int64_t u, int64_t *saddr, int64_t *daddr,
                                int *rr, int *dd, uint64_t *key, int64_t *val, int *err) {
    W_EACH(x, N) {
        int64_t lo = 0, hi = a.E - 1;   // largest in-edge whose first unit is <= x
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (uoff[mid] <= x) lo = mid; else hi = mid - 1;
        }
        const int64_t i = lo, b = (x - uoff[i]) * u;
        const int64_t e = a.match_in[i];
        const int r = a.out_owner[e], d = a.in_owner[i];
        const gbx_datatype_t Ts = a.types[a.sendtypes[e]], Tr = a.types[a.recvtypes[i]];
        const int64_t sa = a.send_base[r] + a.sdispls[e] + wtype_byte(Ts, b);
        const int64_t da = a.recv_base[d] + a.rdispls[i] + wtype_byte(Tr, b);
        if (sa + u > a.send_bytes || da + u > a.recv_bytes) wset_err(err, GBX_ERR_INDEX);
        if ((sa - a.send_base[r]) / u >= (1ll << 31)) wset_err(err, GBX_ERR_UNSUPPORTED);
        saddr[x] = sa;
        daddr[x] = da;
        rr[x] = r;
        dd[x] = d;
        key[x] = (uint64_t)da;
        val[x] = x;
    }
}

__global__ void w_dup_kernel(const uint64_t *key, int64_t n, int *err) {
    W_EACH(m, n) if (m > 0 && key[m] == key[m - 1]) wset_err(err, GBX_ERR_OVERLAP);
}

__global__ void w_order_key_kernel(const int64_t *daddr, const int *dd, int64_t N, int abits, uint64_t *key,
                                   int64_t *val) {
    W_EACH(x, N) {
        key[x] = ((uint64_t)dd[x] << abits) | (uint64_t)daddr[x];
        val[x] = x;
    }
}

// segment starts: a new destination or source rank, or a receive address that does not
// continue the previous unit's
__global__ void w_flag_kernel(const int64_t *ord, const int64_t *daddr, const int *rr, const int *dd, int64_t N,
                              int64_t u, int64_t *flag) {
    W_EACH(m, N) {
        const int64_t x = ord[m];
        int64_t f = 1;
        if (m > 0) {
            const int64_t y = ord[m - 1];
            f = rr[x] != rr[y] || dd[x] != dd[y] || daddr[x] != daddr[y] + u;
        }
        flag[m] = f;
    }
}

__global__ void w_seg_kernel(WArgs a, const int64_t *ord, const int64_t *saddr, const int64_t *daddr, const int *rr,
                             const int *dd, const int64_t *flag, const int64_t *segid, int64_t N, int64_t u,
                             Seg *segs, int64_t *segv0, int *seg_src, int *seg_dst, int32_t *srcel) {
    W_EACH(m, N) {
        const int64_t x = ord[m];
        const int r = rr[x];
        srcel[m] = (int32_t)((saddr[x] - a.send_base[r]) / u);
        if (flag[m]) {
            const int64_t q = segid[m];
            Seg sg;
            sg.v0 = m;
            sg.dst_off = daddr[x];
            sg.src_off = a.send_base[r];
            sg.idx_off = m;
            segs[q] = sg;
            segv0[q] = m;
            seg_src[q] = r;
            seg_dst[q] = dd[x];
        }
    }
}

}  // namespace

int gbx_setup_alltoallw(gbx_request_s *req, const int64_t *send_base, const int *sendcounts, const int64_t *sdispls,
                        const int *sendtypes, const int64_t *recv_base, const int *recvcounts, const int64_t *rdispls,
                        const int *recvtypes, const gbx_datatype_t *types, int ntypes) {
    gbx_graph_s *g = req->graph;
    cudaStream_t st = req->stream;
    const int64_t E = g->E;
    DevPool ws;
    // the datatype table, checked on the host
    unsigned long long talign = 0;
    for (int k = 0; k < ntypes; k++) {
        const gbx_datatype_t &t = types[k];
        if (t.blocklen < 0 || t.extent < 0) return GBX_ERR_ARG;
        int64_t size = t.blocklen;
        for (int l = 0; l < 3; l++) {
            if (t.count[l] < 0 || t.stride[l] < 0) return GBX_ERR_ARG;
            if (t.count[l] > 0 && size > kTypeMaxSize / t.count[l]) return GBX_ERR_ARG;
            size *= t.count[l];
        }
        if (size > kTypeMaxSize) return GBX_ERR_ARG;
        if (size == 0) continue;
        talign |= (unsigned long long)t.blocklen | (unsigned long long)t.extent;
        for (int l = 0; l < 3; l++)
            if (t.count[l] > 1) talign |= (unsigned long long)t.stride[l];
    }
    gbx_datatype_t *d_types = nullptr;
    int *err;
    unsigned long long *align_or;
    int64_t *nbytes;
    GBX_TRY(ws.get(&err, 1));
    GBX_TRY(ws.get(&align_or, 1));
    GBX_TRY(ws.get(&nbytes, E > 0 ? E : 1));
    if (ntypes > 0) {
        GBX_TRY(ws.alloc((void **)&d_types, sizeof(gbx_datatype_t) * ntypes));
        GBX_CUDA_TRY(cudaMemcpyAsync(d_types, types, sizeof(gbx_datatype_t) * ntypes, cudaMemcpyHostToDevice, st));
    }
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    GBX_CUDA_TRY(cudaMemsetAsync(align_or, 0, sizeof(unsigned long long), st));
    WArgs a;
    a.out_owner = g->out_owner; a.in_owner = g->in_owner; a.match_in = g->match_in;
    a.sendcounts = sendcounts; a.sendtypes = sendtypes; a.recvcounts = recvcounts; a.recvtypes = recvtypes;
    a.sdispls = sdispls; a.rdispls = rdispls; a.send_base = send_base; a.recv_base = recv_base;
    a.types = d_types; a.ntypes = ntypes; a.P = g->P;
    a.E = E; a.send_bytes = req->src_bytes; a.recv_bytes = req->dst_bytes;
    w_base_kernel<<<wgrid(g->P), WT, 0, st>>>(a, err, align_or);
    if (E > 0) w_edge_kernel<<<wgrid(E), WT, 0, st>>>(a, nbytes, err, align_or);
    GBX_CUDA_TRY(cudaGetLastError());
    int rc = gbx_read_err(err, st);
    if (rc != 0x7f7f7f7f) return rc;
    unsigned long long h_align = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&h_align, align_or, sizeof(h_align), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    h_align |= talign;
    int64_t u = 16;
    while (u > 1 && (h_align & (unsigned long long)(u - 1))) u >>= 1;
    req->elem_size = u;
    req->align = h_align | (unsigned long long)u | (unsigned long long)(uintptr_t)req->src |
                 (unsigned long long)(uintptr_t)req->dst;

    // units per in-edge, in in-edge order
    int64_t *nunits, *nonzero, *uoff, *nzoff;
    GBX_TRY(ws.get(&nunits, E > 0 ? E : 1));
    GBX_TRY(ws.get(&nonzero, E > 0 ? E : 1));
    GBX_TRY(ws.get(&uoff, E + 1));
    GBX_TRY(ws.get(&nzoff, E + 1));
    int64_t N = 0, nonempty = 0;
    if (E > 0) {
        w_units_kernel<<<wgrid(E), WT, 0, st>>>(nbytes, E, u, nunits, nonzero);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(nunits, uoff, E, st, ws));
        GBX_TRY(gbx_scan_i64(nonzero, nzoff, E, st, ws));
        GBX_TRY(gbx_read_i64(uoff + E, &N, st));
        GBX_TRY(gbx_read_i64(nzoff + E, &nonempty, st));
    }
    const int abits = std::max(1, bitlen_u64((uint64_t)req->dst_bytes));
    const int dbits = std::max(1, bitlen_u64((uint64_t)g->P));
    if (abits + dbits > 64) return GBX_ERR_UNSUPPORTED;

    int64_t nseg = 0;
    Seg *segs = nullptr;
    int64_t *segv0 = nullptr;
    int *seg_src = nullptr, *seg_dst = nullptr;
    int32_t *srcel = nullptr;
    if (N > 0) {
        int64_t *saddr, *daddr, *valA, *valB, *flag, *segid;
        int *rr, *dd;
        uint64_t *keyA, *keyB;
        GBX_TRY(ws.get(&saddr, N)); GBX_TRY(ws.get(&daddr, N));
        GBX_TRY(ws.get(&rr, N)); GBX_TRY(ws.get(&dd, N));
        GBX_TRY(ws.get(&keyA, N)); GBX_TRY(ws.get(&keyB, N));
        GBX_TRY(ws.get(&valA, N)); GBX_TRY(ws.get(&valB, N));
        uint64_t *key = keyA;
        int64_t *val = valA;
        w_expand_kernel<<<wgrid(N), WT, 0, st>>>(a, uoff, N, u, saddr, daddr, rr, dd, key, val, err);
        GBX_CUDA_TRY(cudaGetLastError());
        rc = gbx_read_err(err, st);
        if (rc != 0x7f7f7f7f) return rc;
        // a receive unit written twice
        GBX_TRY(gbx_sort_pairs(&key, &val, keyB, valB, N, abits, st, ws));
        w_dup_kernel<<<wgrid(N), WT, 0, st>>>(key, N, err);
        GBX_CUDA_TRY(cudaGetLastError());
        rc = gbx_read_err(err, st);
        if (rc != 0x7f7f7f7f) return rc;
        // receive order: (destination rank, receive address)
        uint64_t *k2 = keyA;
        int64_t *v2 = valA;
        w_order_key_kernel<<<wgrid(N), WT, 0, st>>>(daddr, dd, N, abits, k2, v2);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&k2, &v2, keyB, valB, N, abits + dbits, st, ws));
        GBX_TRY(ws.get(&flag, N));
        GBX_TRY(ws.get(&segid, N + 1));
        w_flag_kernel<<<wgrid(N), WT, 0, st>>>(v2, daddr, rr, dd, N, u, flag);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(flag, segid, N, st, ws));
        GBX_TRY(gbx_read_i64(segid + N, &nseg, st));
        GBX_TRY(req->mem.get(&segs, nseg));
        GBX_TRY(req->mem.get(&segv0, nseg + 1));
        GBX_TRY(req->mem.get(&seg_src, nseg));
        GBX_TRY(req->mem.get(&seg_dst, nseg));
        GBX_TRY(req->mem.get(&srcel, N));
        w_seg_kernel<<<wgrid(N), WT, 0, st>>>(a, v2, saddr, daddr, rr, dd, flag, segid, N, u, segs, segv0, seg_src,
                                             seg_dst, srcel);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_CUDA_TRY(cudaMemcpyAsync(segv0 + nseg, &N, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        GBX_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        GBX_TRY(req->mem.get(&segv0, 1));
        GBX_CUDA_TRY(cudaMemsetAsync(segv0, 0, sizeof(int64_t), st));
    }
    GBX_TRY(req->mem.get(&req->send_base_copy, g->P));
    GBX_CUDA_TRY(cudaMemcpyAsync(req->send_base_copy, send_base, sizeof(int64_t) * g->P, cudaMemcpyDeviceToDevice, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    req->V = N;
    req->nseg = nseg;
    req->segs_std = segs;
    req->segv0 = segv0;
    req->seg_src_rank = seg_src;
    req->seg_dst_rank = seg_dst;
    req->srcel = srcel;
    req->algorithm = GBX_ALG_STANDARD;
    req->info.V = N;
    req->info.E = E;
    req->info.E_nonzero = nonempty;
    req->info.elem_size = u;
    req->info.user_bytes = 2 * N * u;
    req->info.U = 0;
    if (N > 0)
        GBX_TRY(gbx_make_copy_op(req, 0, req->src, ROLE_SRC, req->dst, ROLE_DST, segs, nseg, srcel, N, N,
                                 2 * N * u + 4 * N + nseg * (int64_t)sizeof(Seg)));
    return GBX_SUCCESS;
}
