// gbx_setup.cu -- device-side setup of the persistent exchange (run once per init).
//
// MPI Advance section 2.2: the persistent neighbourhood collective pays every setup
// cost once, at init, so that start only moves data.  Here that setup runs on the GPU:
//   graph:    CSR and rank validation; MPI multigraph matching of every out-edge with an
//             in-edge (both edge lists stably sorted by (receiver, sender): the t-th
//             listing pairs with the t-th listing);
//   forward:  count / bound / global-index validation, receive-order segments (one per
//             message), per-element source indices (the pack-by-send-list step), the
//             overlap check, and for the locality-aware form (section 1 and section 2.2,
//             last paragraph) the node-pair aggregates: inter-node elements keyed by
//             (node pair, global index), deduplicated, ordered by (node pair,
//             representative rank, global index), plus the step 1 / 2 / 3 descriptors;
//   backward: reverse maps -- per source element, its receive slots in the fixed order
//             (a stable sort of the forward's elements by source offset).
// Errors go to a device word with atomicMin, so the lowest code found wins; the host
// reads it once per stage.  No kernel waits on another block.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "gbx_internal.cuh"

#define SETUP_T 256

static unsigned grid_of(int64_t n) {
    int64_t g = ceil_div(n > 0 ? n : 1, SETUP_T);
    if (g > 65535ll * 32) g = 65535ll * 32;
    return (unsigned)g;
}

#define FOR_EACH(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void set_err(int *err, int code) { atomicMin(err, code); }

// largest i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x)
template <typename T>
__device__ __forceinline__ int64_t upper_index(const T *a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------ graph
__global__ void csr_check_kernel(const int *ptr, int P, int64_t n, int *err) {
    FOR_EACH(r, (int64_t)P + 1) {
        if (r == 0 && ptr[0] != 0) set_err(err, GBX_ERR_ARG);
        if (r == P && (int64_t)ptr[P] != n) set_err(err, GBX_ERR_ARG);
        if (r < P && ptr[r + 1] < ptr[r]) set_err(err, GBX_ERR_ARG);
    }
}

__global__ void rank_check_kernel(const int *ranks, int64_t n, int P, int *err) {
    FOR_EACH(i, n) if (ranks[i] < 0 || ranks[i] >= P) set_err(err, GBX_ERR_RANK);
}

__global__ void owner_kernel(const int *ptr, int P, int64_t n, int *owner) {
    FOR_EACH(e, n) owner[e] = (int)upper_index(ptr, P, e);
}

// key = (receiver << rb) | sender for both edge lists; val = edge index
__global__ void edge_key_kernel(const int *owner, const int *peer, int64_t n, int rb, int owner_is_receiver,
                                uint64_t *keys, int64_t *vals) {
    FOR_EACH(e, n) {
        uint64_t recv = owner_is_receiver ? (uint64_t)owner[e] : (uint64_t)peer[e];
        uint64_t send = owner_is_receiver ? (uint64_t)peer[e] : (uint64_t)owner[e];
        keys[e] = (recv << rb) | send;
        vals[e] = e;
    }
}

__global__ void match_kernel(const uint64_t *ko, const int64_t *vo, const uint64_t *ki, const int64_t *vi,
                             int64_t n, int64_t *match_out, int64_t *match_in, int *err) {
    FOR_EACH(m, n) {
        if (ko[m] != ki[m]) { set_err(err, GBX_ERR_TRUNCATE); continue; }
        match_out[vo[m]] = vi[m];
        match_in[vi[m]] = vo[m];
    }
}

int gbx_graph_setup(gbx_graph_s *g, int64_t n_in, const int *in_ptr, const int *sources,
                    int64_t n_out, const int *out_ptr, const int *dests, cudaStream_t st) {
    const int P = g->P;
    DevPool ws;
    int *err;
    GBX_TRY(ws.get(&err, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));  // 0x7f7f7f7f > any code
    GBX_TRY(g->mem.get(&g->in_ptr, P + 1));
    GBX_TRY(g->mem.get(&g->out_ptr, P + 1));
    GBX_TRY(g->mem.get(&g->sources, n_in));
    GBX_TRY(g->mem.get(&g->dests, n_out));
    GBX_CUDA_TRY(cudaMemcpyAsync(g->in_ptr, in_ptr, sizeof(int) * (P + 1), cudaMemcpyDeviceToDevice, st));
    GBX_CUDA_TRY(cudaMemcpyAsync(g->out_ptr, out_ptr, sizeof(int) * (P + 1), cudaMemcpyDeviceToDevice, st));
    if (n_in) GBX_CUDA_TRY(cudaMemcpyAsync(g->sources, sources, sizeof(int) * n_in, cudaMemcpyDeviceToDevice, st));
    if (n_out) GBX_CUDA_TRY(cudaMemcpyAsync(g->dests, dests, sizeof(int) * n_out, cudaMemcpyDeviceToDevice, st));
    csr_check_kernel<<<grid_of(P + 1), SETUP_T, 0, st>>>(g->in_ptr, P, n_in, err);
    csr_check_kernel<<<grid_of(P + 1), SETUP_T, 0, st>>>(g->out_ptr, P, n_out, err);
    GBX_CUDA_TRY(cudaGetLastError());
    int rc = gbx_read_err(err, st);
    if (rc == 0x7f7f7f7f) rc = GBX_SUCCESS;
    if (rc) return rc;
    if (n_in) rank_check_kernel<<<grid_of(n_in), SETUP_T, 0, st>>>(g->sources, n_in, P, err);
    if (n_out) rank_check_kernel<<<grid_of(n_out), SETUP_T, 0, st>>>(g->dests, n_out, P, err);
    GBX_CUDA_TRY(cudaGetLastError());
    rc = gbx_read_err(err, st);
    if (rc == 0x7f7f7f7f) rc = GBX_SUCCESS;
    if (rc) return rc;
    if (n_in != n_out) return GBX_ERR_TRUNCATE;
    const int64_t E = n_in;
    g->E = E;
    GBX_TRY(g->mem.get(&g->in_owner, E));
    GBX_TRY(g->mem.get(&g->out_owner, E));
    GBX_TRY(g->mem.get(&g->match_out, E));
    GBX_TRY(g->mem.get(&g->match_in, E));
    if (E == 0) return GBX_SUCCESS;
    owner_kernel<<<grid_of(E), SETUP_T, 0, st>>>(g->in_ptr, P, E, g->in_owner);
    owner_kernel<<<grid_of(E), SETUP_T, 0, st>>>(g->out_ptr, P, E, g->out_owner);
    const int rb = std::max(1, bitlen_u64((uint64_t)P - 1));
    uint64_t *ko, *ki, *ka;
    int64_t *vo, *vi, *va;
    GBX_TRY(ws.get(&ko, E)); GBX_TRY(ws.get(&ki, E)); GBX_TRY(ws.get(&ka, E));
    GBX_TRY(ws.get(&vo, E)); GBX_TRY(ws.get(&vi, E)); GBX_TRY(ws.get(&va, E));
    edge_key_kernel<<<grid_of(E), SETUP_T, 0, st>>>(g->out_owner, g->dests, E, rb, 0, ko, vo);
    edge_key_kernel<<<grid_of(E), SETUP_T, 0, st>>>(g->in_owner, g->sources, E, rb, 1, ki, vi);
    GBX_CUDA_TRY(cudaGetLastError());
    uint64_t *ko_s = ko, *ki_s = ki;
    int64_t *vo_s = vo, *vi_s = vi;
    GBX_TRY(gbx_sort_pairs(&ko_s, &vo_s, ka, va, E, 2 * rb, st, ws));
    // second sort needs its own alternate buffers (ka/va may now hold the out result)
    uint64_t *kb; int64_t *vb;
    GBX_TRY(ws.get(&kb, E)); GBX_TRY(ws.get(&vb, E));
    GBX_TRY(gbx_sort_pairs(&ki_s, &vi_s, kb, vb, E, 2 * rb, st, ws));
    match_kernel<<<grid_of(E), SETUP_T, 0, st>>>(ko_s, vo_s, ki_s, vi_s, E, g->match_out, g->match_in, err);
    GBX_CUDA_TRY(cudaGetLastError());
    rc = gbx_read_err(err, st);
    if (rc == 0x7f7f7f7f) rc = GBX_SUCCESS;
    return rc;
}

// ----------------------------------------------------------------- forward setup
struct FwdArgs {
    const int64_t *send_base, *recv_base;
    const int *sendcounts, *sdispls, *recvcounts, *rdispls;
    const int64_t *send_slot_ptr, *recv_slot_ptr;
    const int *send_idx;
    const int64_t *global_sidx, *global_ridx;
    const int *in_owner, *out_owner;
    const int64_t *match_in, *match_out;
    int64_t s, send_bytes, recv_bytes;
    int P, ppn, nnodes;
};

__global__ void base_check_kernel(FwdArgs a, int *err, unsigned long long *align_or) {
    FOR_EACH(r, (int64_t)a.P) {
        if (a.send_base[r] < 0 || a.recv_base[r] < 0) set_err(err, GBX_ERR_INDEX);
        atomicOr(align_or, (unsigned long long)(a.send_base[r] | a.recv_base[r]));
    }
}

// Stage A, per in-edge i: counts, displacements, bounds (the oracle's rules); sort key
// (receiver, rdispl) so that segments come out in receive order.
__global__ void inedge_kernel(FwdArgs a, int64_t E, int64_t *cnt_out, uint64_t *key, int64_t *val, int *err) {
    FOR_EACH(i, E) {
        const int64_t e = a.match_in[i];
        const int r = a.out_owner[e], d = a.in_owner[i];
        const int64_t cnt = a.sendcounts[e];
        const int64_t sd = a.sdispls[e], rd = a.rdispls[i];
        key[i] = ((uint64_t)d << 31) | (uint64_t)(rd >= 0 ? rd : 0);
        val[i] = i;
        cnt_out[i] = 0;
        if ((int64_t)a.recvcounts[i] != cnt || cnt < 0) { set_err(err, GBX_ERR_TRUNCATE); continue; }
        bool ok = true;
        if (sd < 0) ok = false;
        else if (a.send_slot_ptr && sd + cnt > a.send_slot_ptr[r + 1] - a.send_slot_ptr[r]) ok = false;
        if (ok && a.send_base[r] >= 0) {
            if (!a.send_idx && a.send_base[r] + (sd + cnt) * a.s > a.send_bytes) ok = false;
        } else {
            ok = false;
        }
        if (rd < 0) ok = false;
        else if (a.recv_slot_ptr && rd + cnt > a.recv_slot_ptr[d + 1] - a.recv_slot_ptr[d]) ok = false;
        else if (a.recv_base[d] < 0 || a.recv_base[d] + (rd + cnt) * a.s > a.recv_bytes) ok = false;
        if (!ok) { set_err(err, GBX_ERR_INDEX); continue; }
        if (sd + cnt > 0x7fffffffll) { set_err(err, GBX_ERR_UNSUPPORTED); continue; }
        cnt_out[i] = cnt;
    }
}

__global__ void gather_counts_kernel(const int64_t *cnt_by_edge, const int64_t *order, int64_t n, int64_t *c,
                                     int64_t *nz) {
    FOR_EACH(m, n) {
        int64_t x = cnt_by_edge[order[m]];
        c[m] = x;
        nz[m] = x > 0;
    }
}

// Compacts non-empty messages into segments (receive order), fills their descriptors.
__global__ void seg_kernel(FwdArgs a, const int64_t *order, const int64_t *c, const int64_t *v0, const int64_t *nzpos,
                           int64_t n, Seg *segs, int64_t *segv0, int *seg_src, int *seg_dst, int64_t *seg_sd,
                           int64_t *seg_rd, int64_t *seg_of_inedge) {
    FOR_EACH(m, n) {
        const int64_t i = order[m];
        if (c[m] == 0) { seg_of_inedge[i] = -1; continue; }
        const int64_t q = nzpos[m];
        const int64_t e = a.match_in[i];
        const int r = a.out_owner[e], d = a.in_owner[i];
        const int64_t sd = a.sdispls[e], rd = a.rdispls[i];
        Seg sg;
        sg.v0 = v0[m];
        sg.dst_off = a.recv_base[d] + rd * a.s;
        if (a.send_idx) { sg.src_off = a.send_base[r]; sg.idx_off = v0[m]; }
        else { sg.src_off = a.send_base[r] + sd * a.s; sg.idx_off = -1; }
        segs[q] = sg;
        segv0[q] = v0[m];
        seg_src[q] = r;
        seg_dst[q] = d;
        seg_sd[q] = sd;
        seg_rd[q] = rd;
        seg_of_inedge[i] = q;
    }
}

// Stage B, per element: source element index (send list), its bound, and the
// receive-side global index check.
__global__ void elem_kernel(FwdArgs a, const int64_t *segv0, int64_t nseg, const int *seg_src, const int *seg_dst,
                            const int64_t *seg_sd, const int64_t *seg_rd, int64_t V, int32_t *srcel, int *err) {
    FOR_EACH(v, V) {
        const int64_t q = upper_index(segv0, nseg, v);
        const int64_t k = v - segv0[q];
        const int r = seg_src[q], d = seg_dst[q];
        const int64_t slot = seg_sd[q] + k;
        int64_t el = slot;
        if (a.send_idx) {
            el = a.send_idx[a.send_slot_ptr[r] + slot];
            if (el < 0 || a.send_base[r] + (el + 1) * a.s > a.send_bytes) {
                set_err(err, GBX_ERR_INDEX);
                el = 0;
            }
        }
        srcel[v] = (int32_t)el;
        if (a.global_ridx &&
            a.global_ridx[a.recv_slot_ptr[d] + seg_rd[q] + k] != a.global_sidx[a.send_slot_ptr[r] + slot])
            set_err(err, GBX_ERR_GIDX);
    }
}

__global__ void overlap_key_kernel(const Seg *segs, const int64_t *segv0, int64_t nseg, int64_t s, uint64_t *key,
                                   int64_t *val) {
    FOR_EACH(q, nseg) {
        key[q] = (uint64_t)segs[q].dst_off;
        val[q] = (segv0[q + 1] - segv0[q]) * s;   // byte length
    }
}

__global__ void overlap_check_kernel(const uint64_t *key, const int64_t *len, int64_t n, int *err) {
    FOR_EACH(m, n) if (m > 0 && (int64_t)key[m] < (int64_t)key[m - 1] + len[m - 1]) set_err(err, GBX_ERR_OVERLAP);
}

static int read_err_stage(int *err, cudaStream_t st) {
    int rc = gbx_read_err(err, st);
    return rc == 0x7f7f7f7f ? GBX_SUCCESS : rc;
}

// ---------------------------------------------------------------- locality maps
__device__ __forceinline__ int node_sz(int a, int P, int ppn) { int n = P - a * ppn; return n < ppn ? n : ppn; }

__global__ void seg_split_kernel(const int *seg_src, const int *seg_dst, const int64_t *segv0, int64_t nseg, int ppn,
                                 int64_t *c_intra, int64_t *c_inter, int64_t *f_intra, int64_t *f_inter) {
    FOR_EACH(q, nseg) {
        const int64_t c = segv0[q + 1] - segv0[q];
        const bool inter = seg_src[q] / ppn != seg_dst[q] / ppn;
        c_intra[q] = inter ? 0 : c;
        c_inter[q] = inter ? c : 0;
        f_intra[q] = !inter;
        f_inter[q] = inter;
    }
}

// step 0 (intra, standard descriptors renumbered) and step 3 (inter, read the receive
// aggregate through idx3) segments
__global__ void seg03_kernel(const Seg *segs, const int64_t *f_intra, const int64_t *v_intra, const int64_t *p_intra,
                             const int64_t *v_inter, const int64_t *p_inter, int64_t nseg, int64_t r_base,
                             Seg *seg0, Seg *seg3) {
    FOR_EACH(q, nseg) {
        Seg sg = segs[q];
        if (f_intra[q]) {
            sg.v0 = v_intra[q];
            seg0[p_intra[q]] = sg;
        } else {
            Seg t;
            t.v0 = v_inter[q];
            t.dst_off = sg.dst_off;
            t.src_off = r_base;
            t.idx_off = v_inter[q];
            seg3[p_inter[q]] = t;
        }
    }
}

// inter-node elements enumerated in out-edge order (the representative order)
__global__ void out_inter_count_kernel(FwdArgs a, int64_t E, const int64_t *seg_of_inedge, const int64_t *segv0,
                                       int64_t *c) {
    FOR_EACH(e, E) {
        const int64_t q = seg_of_inedge[a.match_out[e]];
        const int r = a.out_owner[e];
        const int d = a.in_owner[a.match_out[e]];
        c[e] = (q >= 0 && r / a.ppn != d / a.ppn) ? segv0[q + 1] - segv0[q] : 0;
    }
}

// gidx of the w-th inter element (out order) and its standard element number
__device__ __forceinline__ void inter_elem(const FwdArgs &a, const int64_t *w0, int64_t E, const int64_t *seg_of_inedge,
                                           const int64_t *segv0, int64_t w, int64_t *v, int64_t *g, int64_t *pair) {
    const int64_t e = upper_index(w0, E, w);
    const int64_t k = w - w0[e];
    const int64_t i = a.match_out[e];
    const int64_t q = seg_of_inedge[i];
    const int r = a.out_owner[e], d = a.in_owner[i];
    *v = segv0[q] + k;
    const int64_t slot = a.sdispls[e] + k;
    if (a.global_sidx) {
        *g = a.global_sidx[a.send_slot_ptr[r] + slot];
    } else {
        // no global indices: a value is named by its source element (its byte offset)
        const int64_t el = a.send_idx ? (int64_t)a.send_idx[a.send_slot_ptr[r] + slot] : slot;
        *g = a.send_base[r] + el * a.s;
    }
    *pair = (int64_t)(r / a.ppn) * a.nnodes + (d / a.ppn);
}

__global__ void gidx_range_kernel(FwdArgs a, const int64_t *w0, int64_t E, const int64_t *seg_of_inedge,
                                  const int64_t *segv0, int64_t W, unsigned long long *mn, unsigned long long *mx) {
    FOR_EACH(w, W) {
        int64_t v, g, pair;
        inter_elem(a, w0, E, seg_of_inedge, segv0, w, &v, &g, &pair);
        unsigned long long u = (unsigned long long)g ^ 0x8000000000000000ull;  // order-preserving
        atomicMin(mn, u);
        atomicMax(mx, u);
    }
}

// mode 0: key = (pair << gbits) | (g - gmin); mode 1: key = g - gmin; val = standard element
__global__ void inter_key_kernel(FwdArgs a, const int64_t *w0, int64_t E, const int64_t *seg_of_inedge,
                                 const int64_t *segv0, int64_t W, int64_t gmin, int gbits, int mode, uint64_t *key,
                                 int64_t *val) {
    FOR_EACH(w, W) {
        int64_t v, g, pair;
        inter_elem(a, w0, E, seg_of_inedge, segv0, w, &v, &g, &pair);
        uint64_t gk = (uint64_t)(g - gmin);
        key[w] = mode == 0 ? (((uint64_t)pair << gbits) | gk) : gk;
        val[w] = w;  // out-order id; converted to the standard element after sorting
    }
}

__global__ void pair_key_kernel(FwdArgs a, const int64_t *w0, int64_t E, const int64_t *seg_of_inedge,
                                const int64_t *segv0, const int64_t *val, int64_t W, uint64_t *key) {
    FOR_EACH(m, W) {
        int64_t v, g, pair;
        inter_elem(a, w0, E, seg_of_inedge, segv0, val[m], &v, &g, &pair);
        key[m] = (uint64_t)pair;
    }
}

// per sorted inter element: (pair, g), new-value flag, and its standard element number
__global__ void value_flag_kernel(FwdArgs a, const int64_t *w0, int64_t E, const int64_t *seg_of_inedge,
                                  const int64_t *segv0, const int64_t *wsorted, int64_t W, int64_t *flag,
                                  int64_t *velem) {
    FOR_EACH(m, W) {
        int64_t v, g, pair;
        inter_elem(a, w0, E, seg_of_inedge, segv0, wsorted[m], &v, &g, &pair);
        velem[m] = v;
        if (m == 0) { flag[m] = 1; continue; }
        int64_t v2, g2, pair2;
        inter_elem(a, w0, E, seg_of_inedge, segv0, wsorted[m - 1], &v2, &g2, &pair2);
        flag[m] = (pair != pair2 || g != g2);
    }
}

// for each distinct value t (at its first sorted occurrence m): aggregate-order key
__global__ void value_rep_kernel(FwdArgs a, const int64_t *flag, const int64_t *tscan, const int64_t *velem,
                                 const int64_t *segv0, int64_t nseg, const int *seg_src, const int *seg_dst,
                                 const int32_t *srcel, int64_t W, int rb, uint64_t *key2, int64_t *val2,
                                 int64_t *rep_off, int32_t *rep_node, int32_t *rep_rank, int32_t *rep_el) {
    FOR_EACH(m, W) {
        if (!flag[m]) continue;
        const int64_t t = tscan[m];
        const int64_t v = velem[m];
        const int64_t q = upper_index(segv0, nseg, v);
        const int r = seg_src[q], d = seg_dst[q];
        const int64_t pair = (int64_t)(r / a.ppn) * a.nnodes + d / a.ppn;
        key2[t] = ((uint64_t)pair << rb) | (uint64_t)r;
        val2[t] = t;
        rep_off[t] = a.send_base[r] + (int64_t)srcel[v] * a.s;
        rep_node[t] = d / a.ppn;
        rep_rank[t] = r;
        rep_el[t] = srcel[v];
    }
}

// aggregate slot arrays (in aggregate order q) and run flags of step 1 / step 2 segments
__global__ void agg_order_kernel(const uint64_t *key2s, const int64_t *tsorted, int64_t U, int rb,
                                 const int64_t *rep_off_t, const int32_t *rep_node_t, const int32_t *rep_el_t,
                                 int64_t *pos_of_t, int64_t *agg_rep_off, int32_t *agg_node, int32_t *idx1,
                                 int64_t *f1, int64_t *f2) {
    FOR_EACH(q, U) {
        const int64_t t = tsorted[q];
        pos_of_t[t] = q;
        agg_rep_off[q] = rep_off_t[t];
        agg_node[q] = rep_node_t[t];
        idx1[q] = rep_el_t[t];
        f1[q] = (q == 0) || key2s[q] != key2s[q - 1];
        f2[q] = (q == 0) || (key2s[q] >> rb) != (key2s[q - 1] >> rb);
    }
}

__global__ void seg12_kernel(FwdArgs a, const uint64_t *key2s, const int64_t *f1, const int64_t *p1,
                             const int64_t *f2, const int64_t *p2, int64_t U, int rb, int64_t r_base,
                             Seg *seg1, Seg *seg2, int64_t *m1) {
    FOR_EACH(q, U) {
        if (f1[q]) {
            const int r = (int)(key2s[q] & ((1ull << rb) - 1));
            const int64_t pair = (int64_t)(key2s[q] >> rb);
            Seg sg;
            sg.v0 = q;
            sg.dst_off = q * a.s;
            sg.src_off = a.send_base[r];
            sg.idx_off = q;
            seg1[p1[q]] = sg;
            const int an = (int)(pair / a.nnodes), bn = (int)(pair % a.nnodes);
            const int lead = an * a.ppn + bn % node_sz(an, a.P, a.ppn);
            if (r != lead) atomicAdd((unsigned long long *)m1, 1ull);
        }
        if (f2[q]) {
            Seg sg;
            sg.v0 = q;
            sg.dst_off = r_base + q * a.s;
            sg.src_off = q * a.s;
            sg.idx_off = -1;
            seg2[p2[q]] = sg;
        }
    }
}

// value id of sorted position m = (inclusive count of first occurrences up to m) - 1
__global__ void idx3_kernel(const int64_t *velem, const int64_t *flag, const int64_t *tscan, const int64_t *pos_of_t,
                            int64_t W, const int64_t *segv0, int64_t nseg, const int64_t *v_inter, int32_t *idx3,
                            int64_t *val_pos) {
    FOR_EACH(m, W) {
        const int64_t v = velem[m];
        const int64_t q = upper_index(segv0, nseg, v);
        const int64_t slot = pos_of_t[tscan[m] + flag[m] - 1];
        idx3[v_inter[q] + (v - segv0[q])] = (int32_t)slot;
        val_pos[v] = slot;
    }
}

// distinct (source node, receiving rank) among inter messages, receiver not the leader
__global__ void m3_key_kernel(const int *seg_src, const int *seg_dst, const int64_t *f_inter, int64_t nseg, int ppn,
                              int nb, uint64_t *key, int64_t *cnt) {
    FOR_EACH(q, nseg) {
        key[q] = f_inter[q] ? (((uint64_t)seg_dst[q] << nb) | (uint64_t)(seg_src[q] / ppn)) : ~0ull;
        cnt[q] = f_inter[q];
    }
}

__global__ void m3_count_kernel(const uint64_t *key, int64_t n, int nb, int P, int ppn, unsigned long long *m3) {
    FOR_EACH(m, n) {
        if (key[m] == ~0ull) continue;
        if (m > 0 && key[m] == key[m - 1]) continue;
        const int d = (int)(key[m] >> nb), an = (int)(key[m] & ((1ull << nb) - 1));
        const int bn = d / ppn;
        const int lead = bn * ppn + an % node_sz(bn, P, ppn);
        if (d != lead) atomicAdd(m3, 1ull);
    }
}

__global__ void fill_i64_neg_kernel(int64_t *p, int64_t n) { FOR_EACH(i, n) p[i] = -1; }

// Receive-order flat index of the locality form's last level: direct elements read the send
// buffer (element index of their source), inter-node elements read the receive aggregate
// (GBX_FLAT_SRC2 | element index in the aggregate buffer).
__global__ void loc_final_index_kernel(const int64_t *segv0, int64_t nseg, const int *seg_src,
                                       const int64_t *send_base, const int32_t *srcel, const int64_t *val_pos,
                                       int64_t V, int64_t s, int64_t U, int32_t *g, int *bad) {
    FOR_EACH(v, V) {
        if (val_pos[v] >= 0) {
            const int64_t el = U + val_pos[v];
            if (el > 0x7fffffffll) { atomicOr(bad, 1); continue; }
            g[v] = (int32_t)(GBX_FLAT_SRC2 | (uint32_t)el);
        } else {
            const int64_t q = upper_index(segv0, nseg, v);
            const int64_t so = send_base[seg_src[q]] + (int64_t)srcel[v] * s;
            if (so % s != 0 || so / s > 0x7fffffffll) { atomicOr(bad, 1); continue; }
            g[v] = (int32_t)(so / s);
        }
    }
}

// --------------------------------------------------------------- forward driver
// -------------------------------------------------------------- debug checks
// GBX_ERR_DUP when an inter-node element's bytes differ from those of the representative of
// its (node pair, global index) value (read from the send buffer at init).
__global__ void dup_check_kernel(const char *src, const int64_t *segv0, int64_t nseg, const int *seg_src,
                                 const int64_t *send_base, const int32_t *srcel, const int64_t *val_pos,
                                 const int64_t *rep_off, int64_t V, int64_t s, int *err) {
    FOR_EACH(v, V) {
        const int64_t q = val_pos[v];
        if (q < 0) continue;
        const int64_t off = send_base[seg_src[upper_index(segv0, nseg, v)]] + (int64_t)srcel[v] * s;
        const int64_t ro = rep_off[q];
        if (off == ro) continue;
        for (int64_t b = 0; b < s; b++)
            if (src[off + b] != src[ro + b]) {
                set_err(err, GBX_ERR_DUP);
                break;
            }
    }
}

// First slot of the receive aggregate: U rounded up to the next count of s-byte slots that
// ends on a 16-byte boundary, so that both halves of the aggregate buffer (send aggregate at
// slot 0, receive aggregate at this slot) start 16-byte aligned and hold the same number of
// slots.  The padding slots are never read by the exchange.
int64_t agg_r_slot(int64_t U, int64_t s) {
    const int64_t m = 16 / std::max<int64_t>(1, std::min<int64_t>(16, s & -s));   // 16 / gcd(s, 16)
    return (U + m - 1) / m * m;
}

// One contiguous segment (copy of the aggregate half at byte offset `from` to the one at
// `to`, element space starting at 0), in device memory owned by `mem`.
static int pair_block_seg(DevPool &mem, int64_t from, int64_t to, cudaStream_t st, Seg **out) {
    Seg h;
    h.v0 = 0;
    h.dst_off = to;
    h.src_off = from;
    h.idx_off = -1;
    GBX_TRY(mem.get(out, 1));
    GBX_CUDA_TRY(cudaMemcpyAsync(*out, &h, sizeof(Seg), cudaMemcpyHostToDevice, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return GBX_SUCCESS;
}

int gbx_setup_forward(gbx_request_s *req, const int64_t *send_base, const int *sendcounts, const int *sdispls,
                      const int64_t *send_slot_ptr, const int *send_idx, const int64_t *recv_base,
                      const int *recvcounts, const int *rdispls, const int64_t *recv_slot_ptr,
                      const int64_t *global_sidx, const int64_t *global_ridx, int want_locality) {
    gbx_graph_s *g = req->graph;
    cudaStream_t st = req->stream;
    const int64_t E = g->E;
    const int64_t s = req->elem_size;
    DevPool ws;
    int *err;
    unsigned long long *align_or;
    GBX_TRY(ws.get(&err, 1));
    GBX_TRY(ws.get(&align_or, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    GBX_CUDA_TRY(cudaMemsetAsync(align_or, 0, sizeof(unsigned long long), st));

    FwdArgs a;
    a.send_base = send_base; a.recv_base = recv_base;
    a.sendcounts = sendcounts; a.sdispls = sdispls; a.recvcounts = recvcounts; a.rdispls = rdispls;
    a.send_slot_ptr = send_slot_ptr; a.recv_slot_ptr = recv_slot_ptr; a.send_idx = send_idx;
    a.global_sidx = global_sidx; a.global_ridx = global_ridx;
    a.in_owner = g->in_owner; a.out_owner = g->out_owner; a.match_in = g->match_in; a.match_out = g->match_out;
    a.s = s; a.send_bytes = req->src_bytes; a.recv_bytes = req->dst_bytes;
    a.P = g->P; a.ppn = g->ppn; a.nnodes = g->nnodes;

    base_check_kernel<<<grid_of(g->P), SETUP_T, 0, st>>>(a, err, align_or);
    GBX_CUDA_TRY(cudaGetLastError());
    int64_t *cnt_e = nullptr, *ordv = nullptr, *ordv_alt = nullptr;
    uint64_t *key = nullptr, *key_alt = nullptr;
    if (E > 0) {
        GBX_TRY(ws.get(&cnt_e, E)); GBX_TRY(ws.get(&key, E)); GBX_TRY(ws.get(&key_alt, E));
        GBX_TRY(ws.get(&ordv, E)); GBX_TRY(ws.get(&ordv_alt, E));
        inedge_kernel<<<grid_of(E), SETUP_T, 0, st>>>(a, E, cnt_e, key, ordv, err);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    GBX_TRY(read_err_stage(err, st));

    // receive order: (receiver, rdispl)
    const int rb = std::max(1, bitlen_u64((uint64_t)g->P - 1));
    int64_t *c = nullptr, *nz = nullptr, *v0 = nullptr, *nzpos = nullptr, *seg_of_inedge = nullptr;
    int64_t nseg = 0, V = 0;
    GBX_TRY(req->mem.get(&seg_of_inedge, E));
    if (E > 0) {
        GBX_TRY(gbx_sort_pairs(&key, &ordv, key_alt, ordv_alt, E, rb + 31, st, ws));
        GBX_TRY(ws.get(&c, E)); GBX_TRY(ws.get(&nz, E));
        GBX_TRY(ws.get(&v0, E + 1)); GBX_TRY(ws.get(&nzpos, E + 1));
        gather_counts_kernel<<<grid_of(E), SETUP_T, 0, st>>>(cnt_e, ordv, E, c, nz);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(c, v0, E, st, ws));
        GBX_TRY(gbx_scan_i64(nz, nzpos, E, st, ws));
        GBX_TRY(gbx_read_i64(v0 + E, &V, st));
        GBX_TRY(gbx_read_i64(nzpos + E, &nseg, st));
    }
    req->V = V;
    req->nseg = nseg;
    int *seg_src, *seg_dst;
    int64_t *seg_sd, *seg_rd, *segv0;
    GBX_TRY(req->mem.get(&req->segs_std, nseg));
    GBX_TRY(req->mem.get(&segv0, nseg + 1));
    GBX_TRY(req->mem.get(&seg_src, nseg));
    GBX_TRY(req->mem.get(&seg_dst, nseg));
    GBX_TRY(ws.get(&seg_sd, nseg));
    GBX_TRY(ws.get(&seg_rd, nseg));
    GBX_TRY(req->mem.get(&req->srcel, V));
    req->seg_src_rank = seg_src;
    req->seg_dst_rank = seg_dst;
    req->segv0 = segv0;
    GBX_TRY(req->mem.get(&req->send_base_copy, g->P));
    GBX_CUDA_TRY(cudaMemcpyAsync(req->send_base_copy, send_base, sizeof(int64_t) * g->P, cudaMemcpyDeviceToDevice, st));
    GBX_CUDA_TRY(cudaMemcpyAsync(segv0 + nseg, &V, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (E > 0) {
        seg_kernel<<<grid_of(E), SETUP_T, 0, st>>>(a, ordv, c, v0, nzpos, E, req->segs_std, segv0, seg_src, seg_dst,
                                                   seg_sd, seg_rd, seg_of_inedge);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    if (V > 0) {
        elem_kernel<<<grid_of(V), SETUP_T, 0, st>>>(a, segv0, nseg, seg_src, seg_dst, seg_sd, seg_rd, V, req->srcel,
                                                    err);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    GBX_TRY(read_err_stage(err, st));
    // receive blocks must not overlap
    if (nseg > 1) {
        uint64_t *ok_, *ok_alt;
        int64_t *ol, *ol_alt;
        GBX_TRY(ws.get(&ok_, nseg)); GBX_TRY(ws.get(&ok_alt, nseg));
        GBX_TRY(ws.get(&ol, nseg)); GBX_TRY(ws.get(&ol_alt, nseg));
        overlap_key_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(req->segs_std, segv0, nseg, s, ok_, ol);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&ok_, &ol, ok_alt, ol_alt, nseg, bitlen_u64((uint64_t)req->dst_bytes), st, ws));
        overlap_check_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(ok_, ol, nseg, err);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(read_err_stage(err, st));
    }
    unsigned long long h_align = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&h_align, align_or, sizeof(h_align), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    h_align |= (unsigned long long)s | (unsigned long long)(uintptr_t)req->src | (unsigned long long)(uintptr_t)req->dst;

    req->align = h_align;

    // the move program
    req->info.V = V;
    req->info.E = E;
    req->info.E_nonzero = nseg;
    req->info.elem_size = s;
    req->info.user_bytes = 2 * V * s;
    // per-message counts: intra / inter split (reported for both forms)
    int64_t *c_intra, *c_inter, *f_intra, *f_inter, *v_intra, *v_inter, *p_intra, *p_inter;
    GBX_TRY(ws.get(&c_intra, nseg)); GBX_TRY(ws.get(&c_inter, nseg));
    GBX_TRY(ws.get(&f_intra, nseg)); GBX_TRY(ws.get(&f_inter, nseg));
    GBX_TRY(ws.get(&v_intra, nseg + 1)); GBX_TRY(ws.get(&v_inter, nseg + 1));
    GBX_TRY(ws.get(&p_intra, nseg + 1)); GBX_TRY(ws.get(&p_inter, nseg + 1));
    int64_t Vd = 0, Vx = 0, n0 = 0, n3 = 0;
    if (nseg > 0) {
        seg_split_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(seg_src, seg_dst, segv0, nseg, g->ppn, c_intra, c_inter,
                                                            f_intra, f_inter);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(c_intra, v_intra, nseg, st, ws));
        GBX_TRY(gbx_scan_i64(c_inter, v_inter, nseg, st, ws));
        GBX_TRY(gbx_scan_i64(f_intra, p_intra, nseg, st, ws));
        GBX_TRY(gbx_scan_i64(f_inter, p_inter, nseg, st, ws));
        GBX_TRY(gbx_read_i64(v_intra + nseg, &Vd, st));
        GBX_TRY(gbx_read_i64(v_inter + nseg, &Vx, st));
        GBX_TRY(gbx_read_i64(p_intra + nseg, &n0, st));
        GBX_TRY(gbx_read_i64(p_inter + nseg, &n3, st));
    }
    req->info.V_direct = Vd;
    req->info.V_inter = Vx;
    req->info.msgs_intra = n0;
    req->info.msgs_inter = n3;
    const int64_t idx_bytes = send_idx ? 4 : 0;

    if (!want_locality) {
        req->algorithm = GBX_ALG_STANDARD;
        if (V > 0)
            GBX_TRY(gbx_make_copy_op(req, 0, req->src, ROLE_SRC, req->dst, ROLE_DST, req->segs_std, nseg,
                                     send_idx ? req->srcel : nullptr, V, V,
                                     2 * V * s + V * idx_bytes + nseg * (int64_t)sizeof(Seg)));
        req->info.U = 0;
        return GBX_SUCCESS;
    }

    // ------------------------------------------------------------ locality form
    req->algorithm = GBX_ALG_LOCALITY;
    Seg *seg0 = nullptr, *seg3 = nullptr;
    GBX_TRY(req->mem.get(&seg0, n0));
    GBX_TRY(req->mem.get(&seg3, n3));
    GBX_TRY(req->mem.get(&req->val_pos, V));
    if (V > 0) {
        fill_i64_neg_kernel<<<grid_of(V), SETUP_T, 0, st>>>(req->val_pos, V);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    // inter elements in out-edge order
    int64_t *c_out, *w0;
    GBX_TRY(ws.get(&c_out, E)); GBX_TRY(ws.get(&w0, E + 1));
    int64_t W = 0;
    if (E > 0) {
        out_inter_count_kernel<<<grid_of(E), SETUP_T, 0, st>>>(a, E, seg_of_inedge, segv0, c_out);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(c_out, w0, E, st, ws));
        GBX_TRY(gbx_read_i64(w0 + E, &W, st));
    }
    if (W != Vx) return GBX_ERR_CUDA;  // internal consistency
    int64_t U = 0, npairs = 0, m1 = 0, m3 = 0, n1 = 0;
    int32_t *idx1 = nullptr, *idx3 = nullptr;
    Seg *seg1 = nullptr, *seg2 = nullptr;
    const int nbits = std::max(1, bitlen_u64((uint64_t)g->nnodes - 1));
    const int pbits = std::max(1, bitlen_u64((uint64_t)g->nnodes * (uint64_t)g->nnodes - 1));
    if (W > 0) {
        unsigned long long *mn, *mx;
        GBX_TRY(ws.get(&mn, 1)); GBX_TRY(ws.get(&mx, 1));
        GBX_CUDA_TRY(cudaMemsetAsync(mn, 0xff, 8, st));
        GBX_CUDA_TRY(cudaMemsetAsync(mx, 0, 8, st));
        gidx_range_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, w0, E, seg_of_inedge, segv0, W, mn, mx);
        GBX_CUDA_TRY(cudaGetLastError());
        unsigned long long hmn = 0, hmx = 0;
        GBX_CUDA_TRY(cudaMemcpyAsync(&hmn, mn, 8, cudaMemcpyDeviceToHost, st));
        GBX_CUDA_TRY(cudaMemcpyAsync(&hmx, mx, 8, cudaMemcpyDeviceToHost, st));
        GBX_CUDA_TRY(cudaStreamSynchronize(st));
        const int64_t gmin = (int64_t)(hmn ^ 0x8000000000000000ull);
        const int64_t gmax = (int64_t)(hmx ^ 0x8000000000000000ull);
        const int gbits = std::max(1, bitlen_u64((uint64_t)(gmax - gmin)));
        uint64_t *k1, *k1a;
        int64_t *w1, *w1a;
        GBX_TRY(ws.get(&k1, W)); GBX_TRY(ws.get(&k1a, W));
        GBX_TRY(ws.get(&w1, W)); GBX_TRY(ws.get(&w1a, W));
        if (pbits + gbits <= 64) {
            inter_key_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, w0, E, seg_of_inedge, segv0, W, gmin, gbits, 0, k1, w1);
            GBX_CUDA_TRY(cudaGetLastError());
            GBX_TRY(gbx_sort_pairs(&k1, &w1, k1a, w1a, W, pbits + gbits, st, ws));
        } else {
            inter_key_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, w0, E, seg_of_inedge, segv0, W, gmin, gbits, 1, k1, w1);
            GBX_CUDA_TRY(cudaGetLastError());
            uint64_t *kk = k1, *kka = k1a;
            int64_t *ww = w1, *wwa = w1a;
            GBX_TRY(gbx_sort_pairs(&kk, &ww, kka, wwa, W, gbits, st, ws));
            uint64_t *kother = (kk == k1) ? k1a : k1;
            int64_t *wother = (ww == w1) ? w1a : w1;
            pair_key_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, w0, E, seg_of_inedge, segv0, ww, W, kk);
            GBX_CUDA_TRY(cudaGetLastError());
            GBX_TRY(gbx_sort_pairs(&kk, &ww, kother, wother, W, pbits, st, ws));
            k1 = kk;
            w1 = ww;
        }
        int64_t *flag, *tscan, *velem;
        GBX_TRY(ws.get(&flag, W)); GBX_TRY(ws.get(&tscan, W + 1)); GBX_TRY(ws.get(&velem, W));
        value_flag_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, w0, E, seg_of_inedge, segv0, w1, W, flag, velem);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(flag, tscan, W, st, ws));
        GBX_TRY(gbx_read_i64(tscan + W, &U, st));
        if (pbits + rb > 64) return GBX_ERR_UNSUPPORTED;
        uint64_t *key2, *key2a;
        int64_t *val2, *val2a, *rep_off, *pos_of_t;
        int32_t *rep_node, *rep_rank, *rep_el;
        GBX_TRY(ws.get(&key2, U)); GBX_TRY(ws.get(&key2a, U));
        GBX_TRY(ws.get(&val2, U)); GBX_TRY(ws.get(&val2a, U));
        GBX_TRY(ws.get(&rep_off, U)); GBX_TRY(ws.get(&pos_of_t, U));
        GBX_TRY(ws.get(&rep_node, U)); GBX_TRY(ws.get(&rep_rank, U)); GBX_TRY(ws.get(&rep_el, U));
        value_rep_kernel<<<grid_of(W), SETUP_T, 0, st>>>(a, flag, tscan, velem, segv0, nseg, seg_src, seg_dst,
                                                         req->srcel, W, rb, key2, val2, rep_off, rep_node, rep_rank,
                                                         rep_el);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&key2, &val2, key2a, val2a, U, pbits + rb, st, ws));
        int64_t *f1, *f2, *p1, *p2;
        GBX_TRY(ws.get(&f1, U)); GBX_TRY(ws.get(&f2, U));
        GBX_TRY(ws.get(&p1, U + 1)); GBX_TRY(ws.get(&p2, U + 1));
        GBX_TRY(req->mem.get(&req->agg_rep_off, U));
        GBX_TRY(req->mem.get(&req->agg_dst_node, U));
        GBX_TRY(req->mem.get(&idx1, U));
        agg_order_kernel<<<grid_of(U), SETUP_T, 0, st>>>(key2, val2, U, rb, rep_off, rep_node, rep_el, pos_of_t,
                                                         req->agg_rep_off, req->agg_dst_node, idx1, f1, f2);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(f1, p1, U, st, ws));
        GBX_TRY(gbx_scan_i64(f2, p2, U, st, ws));
        GBX_TRY(gbx_read_i64(p1 + U, &n1, st));
        GBX_TRY(gbx_read_i64(p2 + U, &npairs, st));
        GBX_TRY(req->mem.get(&seg1, n1));
        GBX_TRY(req->mem.get(&seg2, npairs));
        int64_t *dm1;
        GBX_TRY(ws.get(&dm1, 1));
        GBX_CUDA_TRY(cudaMemsetAsync(dm1, 0, 8, st));
        seg12_kernel<<<grid_of(U), SETUP_T, 0, st>>>(a, key2, f1, p1, f2, p2, U, rb, agg_r_slot(U, s) * s, seg1,
                                                     seg2, dm1);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_read_i64(dm1, &m1, st));
        GBX_TRY(req->mem.get(&idx3, Vx));
        idx3_kernel<<<grid_of(W), SETUP_T, 0, st>>>(velem, flag, tscan, pos_of_t, W, segv0, nseg, v_inter, idx3,
                                                    req->val_pos);
        GBX_CUDA_TRY(cudaGetLastError());
        // step 3 messages
        uint64_t *k3, *k3a;
        int64_t *c3, *c3a;
        GBX_TRY(ws.get(&k3, nseg)); GBX_TRY(ws.get(&k3a, nseg));
        GBX_TRY(ws.get(&c3, nseg)); GBX_TRY(ws.get(&c3a, nseg));
        m3_key_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(seg_src, seg_dst, f_inter, nseg, g->ppn, nbits, k3, c3);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&k3, &c3, k3a, c3a, nseg, 64, st, ws));
        unsigned long long *dm3;
        GBX_TRY(ws.get(&dm3, 1));
        GBX_CUDA_TRY(cudaMemsetAsync(dm3, 0, 8, st));
        m3_count_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(k3, nseg, nbits, g->P, g->ppn, dm3);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_read_i64((const int64_t *)dm3, &m3, st));
        GBX_TRY(req->mem.get(&req->segs_pair, npairs));
        GBX_CUDA_TRY(cudaMemcpyAsync(req->segs_pair, seg2, sizeof(Seg) * npairs, cudaMemcpyDeviceToDevice, st));
    }
    if (nseg > 0) {
        seg03_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(req->segs_std, f_intra, v_intra, p_intra, v_inter, p_inter,
                                                        nseg, agg_r_slot(U, s) * s, seg0, seg3);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    if (req->check_dup && U > 0) {
        // the debug check: one global index per node pair must carry one value
        dup_check_kernel<<<grid_of(V), SETUP_T, 0, st>>>(req->src, segv0, nseg, seg_src, req->send_base_copy,
                                                         req->srcel, req->val_pos, req->agg_rep_off, V, s, err);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(read_err_stage(err, st));
    }
    req->U = U;
    const int64_t Ur = agg_r_slot(U, s);
    req->Ur = Ur;
    req->npairs = npairs;
    req->info.U = U;
    req->info.node_pairs = npairs;
    req->info.msgs_step1 = m1;
    req->info.msgs_step3 = m3;
    if (U > 0) {
        GBX_TRY(req->mem.alloc((void **)&req->agg, (size_t)(2 * Ur * s)));
        GBX_CUDA_TRY(cudaMemsetAsync(req->agg, 0, (size_t)(2 * Ur * s), st));   // (padding slots stay defined)
    }
    // When the receive buffer is one contiguous run in receive order, the direct copies and
    // the redistribution become one receive-order flat op of the last level (each element
    // reads the send buffer or the receive aggregate); otherwise direct copies run in level 0
    // and the redistribution in level 2.
    int combined = 0;
    int32_t *gfin = nullptr;
    int64_t dst0 = 0;
    if (U > 0 && V > 0 && !req->no_combine) {
        int ok = 0;
        int32_t *gtmp = nullptr;
        GBX_TRY(gbx_make_flat(req, req->segs_std, nseg, send_idx ? req->srcel : nullptr, V, &gtmp, &dst0, &ok));
        if (ok) {
            int *bad;
            GBX_TRY(ws.get(&bad, 1));
            GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
            loc_final_index_kernel<<<grid_of(V), SETUP_T, 0, st>>>(segv0, nseg, seg_src, req->send_base_copy,
                                                                   req->srcel, req->val_pos, V, s, Ur, gtmp, bad);
            GBX_CUDA_TRY(cudaGetLastError());
            int hb = 0;
            GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
            GBX_CUDA_TRY(cudaStreamSynchronize(st));
            if (!hb) { combined = 1; gfin = gtmp; }
        }
    }
    if (!combined && n0 > 0)
        GBX_TRY(gbx_make_copy_op(req, 0, req->src, ROLE_SRC, req->dst, ROLE_DST, seg0, n0,
                                 send_idx ? req->srcel : nullptr, V, Vd,
                                 2 * Vd * s + Vd * idx_bytes + n0 * (int64_t)sizeof(Seg)));
    if (U > 0) {
        GBX_TRY(gbx_make_copy_op(req, 0, req->src, ROLE_SRC, req->agg, ROLE_AGG, seg1, n1, idx1, U, U,
                                 2 * U * s + 4 * U));
        // step 2: the node pairs' blocks sit in the same order and at the same offsets in both
        // aggregates, so together they are one contiguous block S -> R (padding slots included)
        Seg *seg2m;
        GBX_TRY(pair_block_seg(req->mem, 0, Ur * s, st, &seg2m));
        GBX_TRY(gbx_make_copy_op(req, 1, req->agg, ROLE_AGG, req->agg, ROLE_AGG, seg2m, 1, nullptr, 0, Ur,
                                 2 * U * s + npairs * (int64_t)sizeof(Seg)));
        if (combined)
            GBX_TRY(gbx_make_flat_op(req, 2, req->src, ROLE_SRC, req->agg, ROLE_AGG, req->dst, ROLE_DST, gfin, V,
                                     dst0));
        else
            GBX_TRY(gbx_make_copy_op(req, 2, req->agg, ROLE_AGG, req->dst, ROLE_DST, seg3, n3, idx3, Vx, Vx,
                                     2 * Vx * s + 4 * Vx + n3 * (int64_t)sizeof(Seg)));
    }
    return GBX_SUCCESS;
}

// -------------------------------------------------------------- backward maps
// standard order: per source element (its byte offset), receive slots in (rank, position)
__global__ void bwd_key_kernel(const int64_t *segv0, int64_t nseg, const int *seg_src, const int32_t *srcel,
                               const int64_t *send_base, int64_t s, int64_t V, uint64_t *key, int64_t *val) {
    FOR_EACH(v, V) {
        const int64_t q = upper_index(segv0, nseg, v);
        key[v] = (uint64_t)(send_base[seg_src[q]] + (int64_t)srcel[v] * s);
        val[v] = v;
    }
}

__global__ void row_flag_kernel(const uint64_t *key, int64_t n, int64_t *flag) {
    FOR_EACH(m, n) flag[m] = (m == 0) || key[m] != key[m - 1];
}

// terms: grad_recv offset of element val[m]; rows: row_ptr / row_out at row starts
__global__ void bwd_terms_kernel(const uint64_t *key, const int64_t *val, const int64_t *flag, const int64_t *rowid,
                                 int64_t n, const Seg *segs, const int64_t *segv0, int64_t nseg, int64_t s,
                                 int64_t out_base, int64_t out_scale, int64_t *terms, int64_t *row_ptr,
                                 int64_t *row_out) {
    FOR_EACH(m, n) {
        const int64_t v = val[m];
        const int64_t q = upper_index(segv0, nseg, v);
        const int64_t off = segs[q].dst_off + (v - segv0[q]) * s;
        terms[m] = off | (flag[m] ? (int64_t)GBX_TERM_GROUP : 0);
        if (flag[m]) {
            row_ptr[rowid[m]] = m;
            row_out[rowid[m]] = out_base + (int64_t)key[m] * out_scale;
        }
    }
}

// node-blocked: reverse step 3 keys (aggregate slot; direct elements sort last)
__global__ void rev3_key_kernel(const int64_t *val_pos, int64_t V, int64_t U, uint64_t *key, int64_t *val) {
    FOR_EACH(v, V) {
        key[v] = val_pos[v] >= 0 ? (uint64_t)val_pos[v] : (uint64_t)U;
        val[v] = v;
    }
}

// node-blocked: records of reverse steps 1 + 0.  Direct element v -> rec v;
// aggregate slot q -> rec V + q.  key = (destination node << obits) | order
__global__ void rev1_key_kernel(const int64_t *val_pos, const int64_t *segv0, int64_t nseg, const int *seg_dst,
                                int64_t V, const int32_t *agg_node, int64_t U, int ppn, int obits, uint64_t sentinel,
                                uint64_t *key, int64_t *val) {
    FOR_EACH(x, V + U) {
        if (x < V) {
            const int64_t q = upper_index(segv0, nseg, x);
            const bool direct = val_pos[x] < 0;
            key[x] = direct ? (((uint64_t)(seg_dst[q] / ppn) << obits) | (uint64_t)x) : sentinel;
        } else {
            key[x] = ((uint64_t)agg_node[x - V] << obits) | (uint64_t)(x - V);
        }
        val[x] = x;
    }
}

__global__ void rev1_srckey_kernel(const int64_t *rec, int64_t n, int64_t V, const int64_t *segv0, int64_t nseg,
                                   const int *seg_src, const int32_t *srcel, const int64_t *send_base, int64_t s,
                                   const int64_t *agg_rep_off, uint64_t *key) {
    FOR_EACH(m, n) {
        const int64_t x = rec[m];
        if (x < V) {
            const int64_t q = upper_index(segv0, nseg, x);
            key[m] = (uint64_t)(send_base[seg_src[q]] + (int64_t)srcel[x] * s);
        } else {
            key[m] = (uint64_t)agg_rep_off[x - V];
        }
    }
}

__global__ void rev1_terms_kernel(const uint64_t *key, const int64_t *rec, const int64_t *rowflag, const int64_t *rowid,
                                  int64_t n, int64_t V, const Seg *segs, const int64_t *segv0, int64_t nseg,
                                  const int *seg_dst, const int32_t *agg_node, int ppn, int64_t s, int64_t *terms,
                                  int64_t *row_ptr, int64_t *row_out) {
    FOR_EACH(m, n) {
        const int64_t x = rec[m];
        int64_t term;
        int node;
        if (x < V) {
            const int64_t q = upper_index(segv0, nseg, x);
            term = segs[q].dst_off + (x - segv0[q]) * s;
            node = seg_dst[q] / ppn;
        } else {
            term = (x - V) * s | (int64_t)GBX_TERM_BUFB;
            node = agg_node[x - V];
        }
        bool gstart = rowflag[m] != 0;
        if (!gstart) {
            const int64_t y = rec[m - 1];
            int pnode;
            if (y < V) pnode = seg_dst[upper_index(segv0, nseg, y)] / ppn;
            else pnode = agg_node[y - V];
            gstart = pnode != node;
        }
        terms[m] = term | (gstart ? (int64_t)GBX_TERM_GROUP : 0);
        if (rowflag[m]) {
            row_ptr[rowid[m]] = m;
            row_out[rowid[m]] = (int64_t)key[m];
        }
    }
}

static int finish_rows(int64_t *row_ptr, int64_t nrows, int64_t nterms, cudaStream_t st) {
    GBX_CUDA_TRY(cudaMemcpyAsync(row_ptr + nrows, &nterms, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return GBX_SUCCESS;
}

int gbx_setup_backward(gbx_request_s *bwd, int accumulate) {
    gbx_request_s *f = bwd->forward;
    cudaStream_t st = bwd->stream;
    const int64_t V = f->V, s = f->elem_size, nseg = f->nseg;
    DevPool ws;
    const int64_t *segv0 = f->segv0;
    const int64_t *send_base = f->send_base_copy;
    const int64_t sbits = std::max(1, bitlen_u64((uint64_t)f->src_bytes));
    bwd->info.V = V;
    bwd->info.E = f->info.E;
    bwd->info.E_nonzero = f->info.E_nonzero;
    bwd->info.elem_size = s;
    bwd->info.user_bytes = 2 * V * s;
    if (V == 0) return GBX_SUCCESS;

    if (f->algorithm == GBX_ALG_STANDARD) {
        uint64_t *k, *ka;
        int64_t *v, *va, *flag, *rowid, *row_ptr, *row_out, *terms;
        GBX_TRY(ws.get(&k, V)); GBX_TRY(ws.get(&ka, V));
        GBX_TRY(ws.get(&v, V)); GBX_TRY(ws.get(&va, V));
        GBX_TRY(ws.get(&flag, V)); GBX_TRY(ws.get(&rowid, V + 1));
        bwd_key_kernel<<<grid_of(V), SETUP_T, 0, st>>>(segv0, nseg, f->seg_src_rank, f->srcel, send_base, s, V, k, v);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&k, &v, ka, va, V, (int)sbits, st, ws));
        row_flag_kernel<<<grid_of(V), SETUP_T, 0, st>>>(k, V, flag);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(flag, rowid, V, st, ws));
        int64_t nrows = 0;
        GBX_TRY(gbx_read_i64(rowid + V, &nrows, st));
        GBX_TRY(bwd->mem.get(&row_ptr, nrows + 1));
        GBX_TRY(bwd->mem.get(&row_out, nrows));
        GBX_TRY(bwd->mem.get(&terms, V + 2));   // 2 entries of padding: the stream fold rounds its copies to 16 bytes
        bwd_terms_kernel<<<grid_of(V), SETUP_T, 0, st>>>(k, v, flag, rowid, V, f->segs_std, segv0, nseg, s, 0, 1,
                                                         terms, row_ptr, row_out);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(finish_rows(row_ptr, nrows, V, st));
        bwd->info.rows = nrows;
        bwd->info.terms = V;
        GBX_TRY(gbx_make_fold_op(bwd, 0, bwd->dst, ROLE_DST, bwd->src, ROLE_SRC, nullptr, ROLE_NONE, row_ptr, row_out,
                                 terms, nrows, V, accumulate));
        return GBX_SUCCESS;
    }

    // node-blocked order: reverse of the three steps
    const int64_t U = f->U, Vx = f->info.V_inter, Vd = f->info.V_direct;
    const int ppn = f->graph->ppn;
    bwd->U = U;
    bwd->npairs = f->npairs;
    bwd->info.U = U;
    bwd->info.node_pairs = f->npairs;
    const int64_t Ur = f->Ur;
    bwd->Ur = Ur;
    if (U > 0) {
        GBX_TRY(bwd->mem.alloc((void **)&bwd->agg, (size_t)(2 * Ur * s)));
        GBX_CUDA_TRY(cudaMemsetAsync(bwd->agg, 0, (size_t)(2 * Ur * s), st));
    }
    int64_t total_terms = 0;
    if (U > 0) {
        // reverse step 3: rows = aggregate slots, terms = their receive slots in (rank, position)
        uint64_t *k, *ka;
        int64_t *v, *va, *flag, *rowid, *row_ptr, *row_out, *terms;
        GBX_TRY(ws.get(&k, V)); GBX_TRY(ws.get(&ka, V));
        GBX_TRY(ws.get(&v, V)); GBX_TRY(ws.get(&va, V));
        GBX_TRY(ws.get(&flag, Vx)); GBX_TRY(ws.get(&rowid, Vx + 1));
        rev3_key_kernel<<<grid_of(V), SETUP_T, 0, st>>>(f->val_pos, V, U, k, v);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&k, &v, ka, va, V, std::max(1, bitlen_u64((uint64_t)U)), st, ws));
        row_flag_kernel<<<grid_of(Vx), SETUP_T, 0, st>>>(k, Vx, flag);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(flag, rowid, Vx, st, ws));
        GBX_TRY(bwd->mem.get(&row_ptr, U + 1));
        GBX_TRY(bwd->mem.get(&row_out, U));
        GBX_TRY(bwd->mem.get(&terms, Vx + 2));
        // rows write the receive-aggregate half (gR) at U*s + slot*s
        bwd_terms_kernel<<<grid_of(Vx), SETUP_T, 0, st>>>(k, v, flag, rowid, Vx, f->segs_std, segv0, nseg, s, Ur * s,
                                                          s, terms, row_ptr, row_out);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(finish_rows(row_ptr, U, Vx, st));
        GBX_TRY(gbx_make_fold_op(bwd, 0, bwd->agg, ROLE_AGG, bwd->src, ROLE_SRC, nullptr, ROLE_NONE, row_ptr, row_out,
                                 terms, U, Vx, 0));
        // reverse step 2: gR -> gS, the node pairs' blocks as one contiguous block
        Seg *rseg2;
        GBX_TRY(pair_block_seg(bwd->mem, Ur * s, 0, st, &rseg2));
        GBX_TRY(gbx_make_copy_op(bwd, 1, bwd->agg, ROLE_AGG, bwd->agg, ROLE_AGG, rseg2, 1, nullptr, 0, Ur,
                                 2 * U * s + f->npairs * (int64_t)sizeof(Seg)));
        total_terms += Vx;
    }
    // reverse steps 1 + 0: rows = source elements; groups by destination node
    {
        const int64_t N = V + U;
        const int obits = std::max(1, bitlen_u64((uint64_t)std::max(V, U)));
        const int nb = std::max(1, bitlen_u64((uint64_t)f->graph->nnodes));
        uint64_t *k, *ka;
        int64_t *x, *xa, *flag, *rowid, *row_ptr, *row_out, *terms;
        GBX_TRY(ws.get(&k, N)); GBX_TRY(ws.get(&ka, N));
        GBX_TRY(ws.get(&x, N)); GBX_TRY(ws.get(&xa, N));
        const uint64_t sentinel = 1ull << (nb + obits);
        rev1_key_kernel<<<grid_of(N), SETUP_T, 0, st>>>(f->val_pos, segv0, nseg, f->seg_dst_rank, V, f->agg_dst_node,
                                                        U, ppn, obits, sentinel, k, x);
        GBX_CUDA_TRY(cudaGetLastError());
        if (nb + obits + 1 > 64) return GBX_ERR_UNSUPPORTED;
        GBX_TRY(gbx_sort_pairs(&k, &x, ka, xa, N, nb + obits + 1, st, ws));
        const int64_t M = Vd + U;   // direct elements and aggregate slots; inter elements sorted last
        uint64_t *sk, *sk_alt;
        int64_t *sx, *sx_alt;
        GBX_TRY(ws.get(&sk, M)); GBX_TRY(ws.get(&sk_alt, M));
        GBX_TRY(ws.get(&sx, M)); GBX_TRY(ws.get(&sx_alt, M));
        if (M > 0) GBX_CUDA_TRY(cudaMemcpyAsync(sx, x, sizeof(int64_t) * M, cudaMemcpyDeviceToDevice, st));
        rev1_srckey_kernel<<<grid_of(M), SETUP_T, 0, st>>>(sx, M, V, segv0, nseg, f->seg_src_rank, f->srcel, send_base,
                                                           s, f->agg_rep_off, sk);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_sort_pairs(&sk, &sx, sk_alt, sx_alt, M, (int)sbits, st, ws));
        GBX_TRY(ws.get(&flag, M)); GBX_TRY(ws.get(&rowid, M + 1));
        row_flag_kernel<<<grid_of(M), SETUP_T, 0, st>>>(sk, M, flag);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(flag, rowid, M, st, ws));
        int64_t nrows = 0;
        GBX_TRY(gbx_read_i64(rowid + M, &nrows, st));
        GBX_TRY(bwd->mem.get(&row_ptr, nrows + 1));
        GBX_TRY(bwd->mem.get(&row_out, nrows));
        GBX_TRY(bwd->mem.get(&terms, M + 2));
        rev1_terms_kernel<<<grid_of(M), SETUP_T, 0, st>>>(sk, sx, flag, rowid, M, V, f->segs_std, segv0, nseg,
                                                          f->seg_dst_rank, f->agg_dst_node, ppn, s, terms, row_ptr,
                                                          row_out);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(finish_rows(row_ptr, nrows, M, st));
        bwd->info.rows = nrows;
        total_terms += M;
        GBX_TRY(gbx_make_fold_op(bwd, U > 0 ? 2 : 0, bwd->dst, ROLE_DST, bwd->src, ROLE_SRC, bwd->agg, ROLE_AGG,
                                 row_ptr, row_out, terms, nrows, M, accumulate));
    }
    bwd->info.terms = total_terms;
    return GBX_SUCCESS;
}

// ------------------------------------------------------- program validation
// Every move program is checked on the device before its first launch: segments strictly
// increasing and non-empty, every destination / source range and every gathered element
// inside its buffer, every fold term and output inside its buffer.  A violation is an
// internal error (GBX_ERR_INTERNAL), reported instead of ever running an out-of-range
// access.
__global__ void check_copy_segs_kernel(const Seg *segs, int64_t nseg, int64_t nelem, int64_t s, int64_t src_bytes,
                                       int64_t dst_bytes, int64_t nidx, int *err) {
    FOR_EACH(q, nseg) {
        const Seg sg = segs[q];
        const int64_t next = q + 1 < nseg ? segs[q + 1].v0 : nelem;
        const int64_t cnt = next - sg.v0;
        bool ok = cnt > 0 && (q > 0 || sg.v0 == 0) && sg.dst_off >= 0 && sg.dst_off + cnt * s <= dst_bytes;
        if (sg.idx_off < 0) ok = ok && sg.src_off >= 0 && sg.src_off + cnt * s <= src_bytes;
        else ok = ok && sg.idx_off + cnt <= nidx && sg.src_off >= 0;
        if (!ok) set_err(err, GBX_ERR_INTERNAL);
    }
}

__global__ void check_copy_idx_kernel(const Seg *segs, int64_t nseg, int64_t nelem, const int32_t *idx, int64_t s,
                                      int64_t src_bytes, int *err) {
    FOR_EACH(v, nelem) {
        int64_t lo = 0, hi = nseg - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (segs[mid].v0 <= v) lo = mid; else hi = mid - 1;
        }
        const Seg sg = segs[lo];
        if (sg.idx_off < 0) continue;
        const int64_t el = idx[sg.idx_off + (v - sg.v0)];
        if (el < 0 || sg.src_off + (el + 1) * s > src_bytes) set_err(err, GBX_ERR_INTERNAL);
    }
}

__global__ void check_fold_kernel(const int64_t *row_ptr, const int64_t *row_out, const longlong2 *rec,
                                  const int64_t *terms, int64_t nrows, int64_t nterms, int64_t s, int64_t out_bytes,
                                  int64_t a_bytes, int64_t b_bytes, int *err) {
    FOR_EACH(r, nrows) {
        const int64_t b = row_ptr[r], e = row_ptr[r + 1];
        bool ok = b < e && (r > 0 || b == 0) && (r + 1 < nrows || e == nterms) && e <= nterms &&
                  row_out[r] >= 0 && row_out[r] + s <= out_bytes;
        const longlong2 x = rec[r];
        if (e - b == 1)
            ok = ok && (uint64_t)x.x == ((uint64_t)row_out[r] | GBX_ROW_SINGLE) && x.y == terms[b];
        else
            ok = ok && x.x == row_out[r] && (uint64_t)x.y == (((uint64_t)b << GBX_ROW_CNT_BITS) | (uint64_t)(e - b));
        for (int64_t m = b; ok && m < e; m++) {
            const uint64_t w = (uint64_t)terms[m];
            const int64_t off = (int64_t)(w & GBX_TERM_MASK);
            const int64_t lim = (w & GBX_TERM_BUFB) ? b_bytes : a_bytes;
            ok = off + s <= lim && (m > b || (w & GBX_TERM_GROUP));
        }
        if (!ok) set_err(err, GBX_ERR_INTERNAL);
    }
}

__global__ void check_flat_kernel(const int32_t *g, int64_t nelem, int64_t s, int64_t dst0, int64_t src_bytes,
                                  int64_t src2_bytes, int64_t dst_bytes, int *err);
__global__ void check_flat2_kernel(const int32_t *gs, const int32_t *gd, int64_t n, int64_t s, int64_t src_bytes,
                                   int64_t src2_bytes, int64_t dst_bytes, int *err);

// ---------------------------------------------------------------- scatter form
// A two-index copy can be read a source window at a time when its element size is a multiple
// of 16 bytes and at most one window, its buffers are 16-byte aligned, and no pair reads the
// second buffer.  The pairs, sorted by source, are grouped by aligned GBX_SCAT_WIN-byte
// window of the source; one thread per window walks its pairs and cuts them into pieces of
// at most GBX_SCAT_RUNS runs and GBX_SCAT_MAXN pairs.  A run is a stretch of source elements
// with no gap longer than GBX_SCAT_GAP bytes: a short gap is cheaper to read than to skip
// with another bulk copy.
__global__ void scatter_flag_kernel(const int32_t *gs, int64_t n, int64_t w, int64_t *flag, int *bad) {
    FOR_EACH(m, n) {
        const uint32_t x = (uint32_t)gs[m];
        if (x & GBX_FLAT_SRC2) *bad = 1;
        if (m > 0 && (uint32_t)gs[m - 1] > x) *bad = 1;   // not in source order
        flag[m] = m == 0 || (int64_t)x / w != (int64_t)(uint32_t)gs[m - 1] / w;
    }
}

__global__ void scatter_start_kernel(const int64_t *flag, const int64_t *pid, int64_t n, int64_t *start) {
    FOR_EACH(m, n) if (flag[m]) start[pid[m]] = m;
}

// Walks window w's pairs; counts its pieces (out == nullptr) or writes them from out[0].
__device__ int64_t scatter_walk(const int32_t *gs, int64_t m0, int64_t m1, int64_t s, ScatterPiece *out) {
    int64_t np = 0;
    ScatterPiece k = {};              // (every field is set at the window's first pair)
    int64_t run_lo = 0, run_hi = 0;   // current run, in source elements [lo, hi]
    auto close_run = [&]() {
        k.run_off[k.nrun] = (uint16_t)((run_lo * s) - k.src);
        k.run_len[k.nrun] = (uint16_t)((run_hi + 1 - run_lo) * s);
        k.nrun++;
        k.len = (int32_t)((run_hi + 1) * s - k.src);
    };
    for (int64_t m = m0; m < m1; m++) {
        const int64_t x = gs[m];
        const bool open = m > m0 && k.n < GBX_SCAT_MAXN;
        if (open && (x - run_hi - 1) * s <= GBX_SCAT_GAP) {   // extends the current run (reading a short gap)
            run_hi = x > run_hi ? x : run_hi;
            k.n++;
            continue;
        }
        if (open && k.nrun + 1 < GBX_SCAT_RUNS) {   // a new run in the same piece
            close_run();
            run_lo = run_hi = x;
            k.n++;
            continue;
        }
        if (m > m0) {   // close the piece
            close_run();
            if (out) out[np] = k;
            np++;
        }
        k.src = x * s;
        k.m0 = m;
        k.n = 1;
        k.nrun = 0;
        k.pad = 0;
        run_lo = run_hi = x;
    }
    if (m1 > m0) {
        close_run();
        if (out) out[np] = k;
        np++;
    }
    return np;
}

__global__ void scatter_count_kernel(const int32_t *gs, const int64_t *start, int64_t nw, int64_t n, int64_t s,
                                     int64_t *cnt) {
    FOR_EACH(w, nw) cnt[w] = scatter_walk(gs, start[w], w + 1 < nw ? start[w + 1] : n, s, nullptr);
}

__global__ void scatter_fill_kernel(const int32_t *gs, const int64_t *start, const int64_t *off, int64_t nw,
                                    int64_t n, int64_t s, ScatterPiece *pieces) {
    FOR_EACH(w, nw) scatter_walk(gs, start[w], w + 1 < nw ? start[w + 1] : n, s, pieces + off[w]);
}

int gbx_make_scatter(gbx_request_s *req, const int32_t *gs, int64_t n, ScatterPiece **pieces,
                     int64_t *npieces, int *ok) {
    cudaStream_t st = req->stream;
    const int64_t s = req->elem_size;
    *ok = 0;
    *npieces = 0;
    if (n <= 0 || (s & 15) || s > GBX_SCAT_WIN || (req->align & 15)) return GBX_SUCCESS;
    DevPool ws;
    int *bad;
    int64_t *flag, *wid, *start, *cnt, *off;
    GBX_TRY(ws.get(&bad, 1));
    GBX_TRY(ws.get(&flag, n));
    GBX_TRY(ws.get(&wid, n + 1));
    GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    scatter_flag_kernel<<<grid_of(n), SETUP_T, 0, st>>>(gs, n, GBX_SCAT_WIN / s, flag, bad);
    GBX_CUDA_TRY(cudaGetLastError());
    int hb = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return GBX_SUCCESS;
    GBX_TRY(gbx_scan_i64(flag, wid, n, st, ws));
    int64_t nw = 0, np = 0;
    GBX_TRY(gbx_read_i64(wid + n, &nw, st));
    GBX_TRY(ws.get(&start, nw));
    GBX_TRY(ws.get(&cnt, nw));
    GBX_TRY(ws.get(&off, nw + 1));
    scatter_start_kernel<<<grid_of(n), SETUP_T, 0, st>>>(flag, wid, n, start);
    GBX_CUDA_TRY(cudaGetLastError());
    scatter_count_kernel<<<grid_of(nw), SETUP_T, 0, st>>>(gs, start, nw, n, s, cnt);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(cnt, off, nw, st, ws));
    GBX_TRY(gbx_read_i64(off + nw, &np, st));
    GBX_TRY(req->mem.get(pieces, np));
    scatter_fill_kernel<<<grid_of(nw), SETUP_T, 0, st>>>(gs, start, off, nw, n, s, *pieces);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    GBX_TRY(gbx_scatter_prepare());
    *npieces = np;
    *ok = 1;
    return GBX_SUCCESS;
}

// every piece inside the source and at most one window, its runs aligned, ascending and
// disjoint inside it, its pairs inside the index arrays; every pair's source inside one of
// its piece's runs and its destination inside the destination
__global__ void check_scatter_kernel(const ScatterPiece *pieces, int64_t np, const int32_t *gs, const int32_t *gd,
                                     int64_t n, int64_t s, int64_t src_bytes, int64_t dst_bytes, int *err) {
    FOR_EACH(p, np) {
        const ScatterPiece k = pieces[p];
        bool good = k.len > 0 && k.len <= GBX_SCAT_WIN && (k.src & 15) == 0 && k.src >= 0 &&
                    k.src + k.len <= src_bytes && k.m0 >= 0 && k.n > 0 && k.n <= GBX_SCAT_MAXN && k.m0 + k.n <= n &&
                    k.nrun > 0 && k.nrun <= GBX_SCAT_RUNS && ((uintptr_t)gs & 15) == 0 && ((uintptr_t)gd & 15) == 0;
        int64_t end = 0;
        for (int r = 0; good && r < k.nrun; r++) {
            const int64_t o = k.run_off[r], l = k.run_len[r];
            good = (o & 15) == 0 && (l & 15) == 0 && l > 0 && o >= end && o + l <= k.len;
            end = o + l;
        }
        int r = 0;
        for (int64_t m = k.m0; good && m < k.m0 + k.n; m++) {
            const int64_t a = (int64_t)(uint32_t)gs[m] * s - k.src;
            while (r < k.nrun && a >= k.run_off[r] + k.run_len[r]) r++;
            good = r < k.nrun && a >= k.run_off[r] && a + s <= k.run_off[r] + k.run_len[r] && gd[m] >= 0 &&
                   ((int64_t)gd[m] + 1) * s <= dst_bytes;
        }
        if (!good) set_err(err, GBX_ERR_INTERNAL);
    }
}

__global__ void check_bulk_kernel(const BulkTask *tasks, int64_t n, int64_t src_bytes, int64_t dst_bytes, int *err) {
    FOR_EACH(m, n) {
        const BulkTask k = tasks[m];
        if (k.len <= 0 || k.len > GBX_BULK_BYTES || (k.len & 15) || (k.src & 15) || (k.dst & 15) || k.src < 0 ||
            k.dst < 0 || k.src + k.len > src_bytes || k.dst + k.len > dst_bytes)
            set_err(err, GBX_ERR_INTERNAL);
    }
}

int gbx_validate_program(gbx_request_s *req, int64_t agg_bytes) {
    cudaStream_t st = req->stream;
    DevPool ws;
    int *err;
    GBX_TRY(ws.get(&err, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    auto bytes_of = [&](int role) -> int64_t {
        return role == ROLE_SRC ? req->src_bytes : role == ROLE_DST ? req->dst_bytes : role == ROLE_AGG ? agg_bytes : 0;
    };
    for (HostOp &op : req->ops) {
        if (op.kind == 0) {
            const CopyDesc &d = op.cd;
            const int64_t nidx = d.idx ? op.idx_len : 0;
            check_copy_segs_kernel<<<grid_of(d.nseg), SETUP_T, 0, st>>>(d.segs, d.nseg, d.nelem, d.elem_size,
                                                                        bytes_of(d.src_role), bytes_of(d.dst_role),
                                                                        nidx, err);
            if (d.idx)
                check_copy_idx_kernel<<<grid_of(d.nelem), SETUP_T, 0, st>>>(d.segs, d.nseg, d.nelem, d.idx,
                                                                            d.elem_size, bytes_of(d.src_role), err);
            if (op.bulk_ok)
                check_bulk_kernel<<<grid_of(op.nbulk), SETUP_T, 0, st>>>(op.d_bulk, op.nbulk, bytes_of(d.src_role),
                                                                         bytes_of(d.dst_role), err);
            if (op.scat_ok)
                check_scatter_kernel<<<grid_of(op.nscat), SETUP_T, 0, st>>>(
                    op.d_scat, op.nscat, d.flat_idx, d.flat_didx, d.nelem, d.elem_size, bytes_of(d.src_role),
                    bytes_of(d.dst_role), err);
            if (op.flat_ok && (d.flat & 3) == 3)
                check_flat2_kernel<<<grid_of(d.nelem), SETUP_T, 0, st>>>(d.flat_idx, d.flat_didx, d.nelem, d.elem_size,
                                                                         bytes_of(d.src_role),
                                                                         d.src2 ? bytes_of(d.src2_role) : 0,
                                                                         bytes_of(d.dst_role), err);
            else if (op.flat_ok)
                check_flat_kernel<<<grid_of(d.nelem), SETUP_T, 0, st>>>(op.d_flat_idx, d.nelem, d.elem_size,
                                                                        op.flat_dst0, bytes_of(d.src_role),
                                                                        d.src2 ? bytes_of(d.src2_role) : 0,
                                                                        bytes_of(d.dst_role), err);
        } else {
            const FoldDesc &d = op.fd;
            check_fold_kernel<<<grid_of(d.nrows), SETUP_T, 0, st>>>(d.row_ptr, d.row_out, d.rec, d.terms, d.nrows,
                                                                    op.idx_len, d.elem_size, bytes_of(d.out_role),
                                                                    bytes_of(d.a_role), bytes_of(d.b_role), err);
        }
        GBX_CUDA_TRY(cudaGetLastError());
    }
    return read_err_stage(err, st);
}

// packed row records of a fold op (see GBX_ROW_SINGLE)
__global__ void fold_rec_kernel(const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms, int64_t nrows,
                                longlong2 *rec, int *err) {
    FOR_EACH(r, nrows) {
        const int64_t b = row_ptr[r], n = row_ptr[r + 1] - b;
        longlong2 x;
        if (n == 1) {
            x.x = (long long)((uint64_t)row_out[r] | GBX_ROW_SINGLE);
            x.y = terms[b];
        } else {
            x.x = row_out[r];
            x.y = (long long)(((uint64_t)b << GBX_ROW_CNT_BITS) | (uint64_t)n);
            if (n <= 0 || n >= (1ll << GBX_ROW_CNT_BITS) || b >= (1ll << (64 - GBX_ROW_CNT_BITS)))
                set_err(err, GBX_ERR_UNSUPPORTED);
        }
        rec[r] = x;
    }
}

int gbx_build_fold_records(const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms, int64_t nrows,
                           longlong2 *rec, cudaStream_t st) {
    DevPool ws;
    int *err;
    GBX_TRY(ws.get(&err, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    fold_rec_kernel<<<grid_of(nrows), SETUP_T, 0, st>>>(row_ptr, row_out, terms, nrows, rec, err);
    GBX_CUDA_TRY(cudaGetLastError());
    return read_err_stage(err, st);
}

// ------------------------------------------------------------ run splitting
// Re-cuts the segments of a gathering copy op so that every run of >= min_run elements
// whose source indices are consecutive becomes a contiguous segment (its elements need
// no index load, so the data load no longer waits for one), while stretches of shorter
// runs stay index-gathered.  The element numbering, the destinations and the bytes moved
// are unchanged.
__device__ __forceinline__ int64_t seg_of(const Seg *segs, int64_t nseg, int64_t v) {
    int64_t lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (segs[mid].v0 <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void run_start_kernel(const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem, int64_t *rs) {
    FOR_EACH(v, nelem) {
        const int64_t q = seg_of(segs, nseg, v);
        const Seg sg = segs[q];
        const int64_t k = v - sg.v0;
        rs[v] = (k == 0) || (sg.idx_off >= 0 && idx[sg.idx_off + k] != idx[sg.idx_off + k - 1] + 1);
    }
}

// run r begins at element begin[r]; a run is long if it has >= min_run elements or lies in
// a segment that was already contiguous
__global__ void run_begin_kernel(const int64_t *rs, const int64_t *rid, int64_t nelem, int64_t *begin) {
    FOR_EACH(v, nelem) if (rs[v]) begin[rid[v]] = v;
}

__global__ void run_long_kernel(const Seg *segs, int64_t nseg, const int64_t *begin, int64_t nruns, int64_t nelem,
                                int min_run, int64_t *is_long) {
    FOR_EACH(r, nruns) {
        const int64_t end = r + 1 < nruns ? begin[r + 1] : nelem;
        const Seg sg = segs[seg_of(segs, nseg, begin[r])];
        is_long[r] = sg.idx_off < 0 || end - begin[r] >= min_run;
    }
}

__global__ void new_seg_flag_kernel(const Seg *segs, int64_t nseg, const int64_t *rs, const int64_t *rid,
                                    const int64_t *is_long, int64_t nelem, int64_t *ns) {
    FOR_EACH(v, nelem) {
        const int64_t q = seg_of(segs, nseg, v);
        const int64_t run = rid[v] + rs[v] - 1;
        ns[v] = (v == segs[q].v0) || (rs[v] && (is_long[run] || is_long[run - 1]));
    }
}

__global__ void new_seg_kernel(const Seg *segs, int64_t nseg, const int32_t *idx, const int64_t *rs, const int64_t *rid,
                               const int64_t *is_long, const int64_t *ns, const int64_t *nsid, int64_t nelem, int64_t s,
                               Seg *out) {
    FOR_EACH(v, nelem) {
        if (!ns[v]) continue;
        const Seg sg = segs[seg_of(segs, nseg, v)];
        const int64_t k = v - sg.v0;
        const int64_t run = rid[v] + rs[v] - 1;
        Seg t;
        t.v0 = v;
        t.dst_off = sg.dst_off + k * s;
        if (sg.idx_off < 0) {
            t.src_off = sg.src_off + k * s;
            t.idx_off = -1;
        } else if (is_long[run]) {
            t.src_off = sg.src_off + (int64_t)idx[sg.idx_off + k] * s;
            t.idx_off = -1;
        } else {
            t.src_off = sg.src_off;
            t.idx_off = sg.idx_off + k;
        }
        out[nsid[v]] = t;
    }
}

int gbx_split_runs(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                   int min_run, Seg **out, int64_t *out_nseg) {
    cudaStream_t st = req->stream;
    DevPool ws;
    int64_t *rs, *rid, *begin, *is_long, *ns, *nsid;
    GBX_TRY(ws.get(&rs, nelem)); GBX_TRY(ws.get(&rid, nelem + 1));
    run_start_kernel<<<grid_of(nelem), SETUP_T, 0, st>>>(segs, nseg, idx, nelem, rs);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(rs, rid, nelem, st, ws));
    int64_t nruns = 0;
    GBX_TRY(gbx_read_i64(rid + nelem, &nruns, st));
    GBX_TRY(ws.get(&begin, nruns)); GBX_TRY(ws.get(&is_long, nruns));
    run_begin_kernel<<<grid_of(nelem), SETUP_T, 0, st>>>(rs, rid, nelem, begin);
    run_long_kernel<<<grid_of(nruns), SETUP_T, 0, st>>>(segs, nseg, begin, nruns, nelem, min_run, is_long);
    GBX_TRY(ws.get(&ns, nelem)); GBX_TRY(ws.get(&nsid, nelem + 1));
    new_seg_flag_kernel<<<grid_of(nelem), SETUP_T, 0, st>>>(segs, nseg, rs, rid, is_long, nelem, ns);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(ns, nsid, nelem, st, ws));
    int64_t n = 0;
    GBX_TRY(gbx_read_i64(nsid + nelem, &n, st));
    Seg *o;
    GBX_TRY(req->mem.get(&o, n));
    new_seg_kernel<<<grid_of(nelem), SETUP_T, 0, st>>>(segs, nseg, idx, rs, rid, is_long, ns, nsid, nelem,
                                                       req->elem_size, o);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    *out = o;
    *out_nseg = n;
    return GBX_SUCCESS;
}

// ------------------------------------------------------- source-ordered pieces
// Cuts every segment into pieces of at most max_piece elements and renumbers the op's
// element space so that pieces come in ascending source address.  Reads that are close in
// memory (for a stencil, the two x faces of a rank, 1984 bytes apart) are then issued
// together, while every piece still writes one contiguous run.  Same elements, same bytes.
__global__ void piece_count_kernel(const Seg *segs, int64_t nseg, int64_t nelem, int64_t max_piece, int64_t *np) {
    FOR_EACH(q, nseg) {
        const int64_t c = (q + 1 < nseg ? segs[q + 1].v0 : nelem) - segs[q].v0;
        np[q] = (c + max_piece - 1) / max_piece;
    }
}

__global__ void piece_make_kernel(const Seg *segs, int64_t nseg, int64_t nelem, int64_t max_piece, const int64_t *pstart,
                                  const int32_t *idx, int64_t s, Seg *pieces, int64_t *len, uint64_t *key, int64_t *pid) {
    FOR_EACH(q, nseg) {
        const Seg sg = segs[q];
        const int64_t c = (q + 1 < nseg ? segs[q + 1].v0 : nelem) - sg.v0;
        for (int64_t j = 0; j * max_piece < c; j++) {
            const int64_t p = pstart[q] + j, k = j * max_piece;
            Seg t;
            t.v0 = 0;
            t.dst_off = sg.dst_off + k * s;
            if (sg.idx_off < 0) { t.src_off = sg.src_off + k * s; t.idx_off = -1; }
            else { t.src_off = sg.src_off; t.idx_off = sg.idx_off + k; }
            pieces[p] = t;
            len[p] = c - k < max_piece ? c - k : max_piece;
            key[p] = (uint64_t)(t.idx_off < 0 ? t.src_off : t.src_off + (int64_t)idx[t.idx_off] * s);
            pid[p] = p;
        }
    }
}

__global__ void piece_gather_len_kernel(const int64_t *len, const int64_t *order, int64_t n, int64_t *olen) {
    FOR_EACH(m, n) olen[m] = len[order[m]];
}

__global__ void piece_place_kernel(const Seg *pieces, const int64_t *order, const int64_t *v0, int64_t n, Seg *out) {
    FOR_EACH(m, n) {
        Seg t = pieces[order[m]];
        t.v0 = v0[m];
        out[m] = t;
    }
}

int gbx_order_by_source(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                        int64_t src_bytes, int64_t max_piece, Seg **out, int64_t *out_nseg) {
    cudaStream_t st = req->stream;
    DevPool ws;
    int64_t *np, *pstart;
    GBX_TRY(ws.get(&np, nseg)); GBX_TRY(ws.get(&pstart, nseg + 1));
    piece_count_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(segs, nseg, nelem, max_piece, np);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(np, pstart, nseg, st, ws));
    int64_t n = 0;
    GBX_TRY(gbx_read_i64(pstart + nseg, &n, st));
    Seg *pieces, *o;
    int64_t *len, *pid, *pida, *olen, *v0;
    uint64_t *key, *keya;
    GBX_TRY(ws.get(&pieces, n)); GBX_TRY(ws.get(&len, n)); GBX_TRY(ws.get(&olen, n)); GBX_TRY(ws.get(&v0, n + 1));
    GBX_TRY(ws.get(&key, n)); GBX_TRY(ws.get(&keya, n)); GBX_TRY(ws.get(&pid, n)); GBX_TRY(ws.get(&pida, n));
    piece_make_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(segs, nseg, nelem, max_piece, pstart, idx, req->elem_size,
                                                         pieces, len, key, pid);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_sort_pairs(&key, &pid, keya, pida, n, std::max(1, bitlen_u64((uint64_t)src_bytes)), st, ws));
    piece_gather_len_kernel<<<grid_of(n), SETUP_T, 0, st>>>(len, pid, n, olen);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(olen, v0, n, st, ws));
    GBX_TRY(req->mem.get(&o, n));
    piece_place_kernel<<<grid_of(n), SETUP_T, 0, st>>>(pieces, pid, v0, n, o);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    *out = o;
    *out_nseg = n;
    return GBX_SUCCESS;
}

// ------------------------------------------------------------------ flat form
// A copy op whose destinations form one contiguous run (every segment starts where the
// previous one ended) and whose source offsets are all multiples of the element size can
// run as a plain indexed gather, dst[e] = src[g[e]], with no segment search.
__global__ void flat_dst_kernel(const Seg *segs, int64_t nseg, int64_t s, int *bad) {
    FOR_EACH(q, nseg) if (segs[q].dst_off != segs[0].dst_off + segs[q].v0 * s) atomicOr(bad, 1);
}

__global__ void flat_build_kernel(const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem, int64_t s,
                                  int32_t *g, int *bad) {
    FOR_EACH(v, nelem) {
        const Seg sg = segs[seg_of(segs, nseg, v)];
        const int64_t k = v - sg.v0;
        const int64_t so = sg.src_off + (sg.idx_off >= 0 ? (int64_t)idx[sg.idx_off + k] : k) * s;
        if (so % s != 0 || so / s > 0x7fffffffll) { atomicOr(bad, 1); continue; }
        g[v] = (int32_t)(so / s);
    }
}

// ------------------------------------------------------------------ bulk form
// An op can move as bulk pieces when every segment is contiguous on both sides and its
// offsets and byte length are multiples of 16; each segment is cut into pieces of at most
// GBX_BULK_BYTES.
__global__ void bulk_count_kernel(const Seg *segs, int64_t nseg, int64_t nelem, int64_t s, int64_t *npieces,
                                  int *bad) {
    FOR_EACH(q, nseg) {
        const int64_t n = (q + 1 < nseg ? segs[q + 1].v0 : nelem) - segs[q].v0;
        const int64_t bytes = n * s;
        if (segs[q].idx_off >= 0 || (segs[q].src_off & 15) || (segs[q].dst_off & 15) || (bytes & 15)) *bad = 1;
        npieces[q] = (bytes + GBX_BULK_BYTES - 1) / GBX_BULK_BYTES;
    }
}

__global__ void bulk_fill_kernel(const Seg *segs, int64_t nseg, int64_t nelem, int64_t s, const int64_t *first,
                                 BulkTask *tasks) {
    FOR_EACH(q, nseg) {
        const int64_t bytes = ((q + 1 < nseg ? segs[q + 1].v0 : nelem) - segs[q].v0) * s;
        for (int64_t m = 0, off = 0; off < bytes; m++, off += GBX_BULK_BYTES) {
            BulkTask k;
            k.src = segs[q].src_off + off;
            k.dst = segs[q].dst_off + off;
            k.len = bytes - off < GBX_BULK_BYTES ? bytes - off : GBX_BULK_BYTES;
            tasks[first[q] + m] = k;
        }
    }
}

// owned: source and destination are the library's own aggregate buffers (256-byte aligned
// allocations), so only the pieces' offsets and lengths decide; otherwise the caller's buffers'
// alignment (and the element size) must be a multiple of 16 as well.
int gbx_make_bulk(gbx_request_s *req, const Seg *segs, int64_t nseg, int64_t nelem, bool owned, BulkTask **out,
                  int64_t *n, int *ok) {
    cudaStream_t st = req->stream;
    *ok = 0;
    *n = 0;
    if (nseg <= 0 || nelem <= 0 || (!owned && (req->align & 15))) return GBX_SUCCESS;
    DevPool ws;
    int *bad;
    int64_t *np, *first;
    GBX_TRY(ws.get(&bad, 1));
    GBX_TRY(ws.get(&np, nseg));
    GBX_TRY(ws.get(&first, nseg + 1));
    GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    bulk_count_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(segs, nseg, nelem, req->elem_size, np, bad);
    GBX_CUDA_TRY(cudaGetLastError());
    int hb = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return GBX_SUCCESS;
    GBX_TRY(gbx_scan_i64(np, first, nseg, st, ws));
    GBX_TRY(gbx_read_i64(first + nseg, n, st));
    GBX_TRY(req->mem.get(out, *n));
    bulk_fill_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(segs, nseg, nelem, req->elem_size, first, *out);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_bulk_prepare());
    *ok = 1;
    return GBX_SUCCESS;
}

int gbx_make_flat(gbx_request_s *req, const Seg *segs, int64_t nseg, const int32_t *idx, int64_t nelem,
                  int32_t **flat_idx, int64_t *dst0, int *ok) {
    cudaStream_t st = req->stream;
    *ok = 0;
    DevPool ws;
    int *bad;
    GBX_TRY(ws.get(&bad, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    flat_dst_kernel<<<grid_of(nseg), SETUP_T, 0, st>>>(segs, nseg, req->elem_size, bad);
    GBX_CUDA_TRY(cudaGetLastError());
    int hb = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return GBX_SUCCESS;
    int32_t *g;
    GBX_TRY(req->mem.get(&g, nelem + 4));   // 4 entries of padding for the stream form's rounded copies
    flat_build_kernel<<<grid_of(nelem), SETUP_T, 0, st>>>(segs, nseg, idx, nelem, req->elem_size, g, bad);
    GBX_CUDA_TRY(cudaGetLastError());
    Seg first;
    GBX_CUDA_TRY(cudaMemcpyAsync(&first, segs, sizeof(Seg), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return GBX_SUCCESS;   // g stays allocated with the request; the flat form is unused
    *flat_idx = g;
    *dst0 = first.dst_off;
    *ok = 1;
    return GBX_SUCCESS;
}

__global__ void check_flat_kernel(const int32_t *g, int64_t nelem, int64_t s, int64_t dst0, int64_t src_bytes,
                                  int64_t src2_bytes, int64_t dst_bytes, int *err) {
    FOR_EACH(v, nelem) {
        const uint32_t x = (uint32_t)g[v];
        const int64_t el = (int64_t)(x & ~GBX_FLAT_SRC2);
        const int64_t lim = (x & GBX_FLAT_SRC2) ? src2_bytes : src_bytes;
        if ((el + 1) * s > lim || dst0 < 0 || dst0 + (v + 1) * s > dst_bytes) set_err(err, GBX_ERR_INTERNAL);
    }
}

// ------------------------------------------------ single-term rows of a fold
// When a fold does not accumulate, a row with one term is a copy out[row] = term: those rows
// become a two-index flat copy and only rows with several terms stay in the fold.  Needs
// every offset to be a multiple of the element size below 2^31 elements (else ok = 0).
__global__ void row_kind_kernel(const int64_t *row_ptr, int64_t nrows, int64_t *single, int64_t *multi,
                                int64_t *mcnt) {
    FOR_EACH(r, nrows) {
        const int64_t c = row_ptr[r + 1] - row_ptr[r];
        single[r] = c == 1;
        multi[r] = c > 1;
        mcnt[r] = c > 1 ? c : 0;
    }
}

__global__ void row_split_kernel(const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms, int64_t nrows,
                                 int64_t s, const int64_t *sidx, const int64_t *mrow, const int64_t *mterm,
                                 int32_t *gs, int32_t *gd, int64_t *row_ptr2, int64_t *row_out2, int64_t *terms2,
                                 int *bad) {
    FOR_EACH(r, nrows) {
        const int64_t b = row_ptr[r], c = row_ptr[r + 1] - b;
        if (c == 1) {
            const uint64_t w = (uint64_t)terms[b];
            const int64_t off = (int64_t)(w & GBX_TERM_MASK);
            if (off % s || row_out[r] % s || off / s > 0x7fffffffll || row_out[r] / s > 0x7fffffffll) {
                atomicOr(bad, 1);
                continue;
            }
            gs[sidx[r]] = (int32_t)(((w & GBX_TERM_BUFB) ? GBX_FLAT_SRC2 : 0u) | (uint32_t)(off / s));
            gd[sidx[r]] = (int32_t)(row_out[r] / s);
        } else {
            const int64_t m = mrow[r], t0 = mterm[r];
            row_ptr2[m] = t0;
            row_out2[m] = row_out[r];
            for (int64_t k = 0; k < c; k++) terms2[t0 + k] = terms[b + k];
        }
    }
}

int gbx_split_single_rows(gbx_request_s *req, const int64_t *row_ptr, const int64_t *row_out, const int64_t *terms,
                          int64_t nrows, int32_t **gs, int32_t **gd, int64_t *nsingle, int64_t **row_ptr2,
                          int64_t **row_out2, int64_t **terms2, int64_t *nmulti, int64_t *nmterms, int *ok) {
    cudaStream_t st = req->stream;
    *ok = 0;
    DevPool ws;
    int64_t *single, *multi, *mcnt, *sidx, *mrow, *mterm;
    int *bad;
    GBX_TRY(ws.get(&single, nrows)); GBX_TRY(ws.get(&multi, nrows)); GBX_TRY(ws.get(&mcnt, nrows));
    GBX_TRY(ws.get(&sidx, nrows + 1)); GBX_TRY(ws.get(&mrow, nrows + 1)); GBX_TRY(ws.get(&mterm, nrows + 1));
    GBX_TRY(ws.get(&bad, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    row_kind_kernel<<<grid_of(nrows), SETUP_T, 0, st>>>(row_ptr, nrows, single, multi, mcnt);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(single, sidx, nrows, st, ws));
    GBX_TRY(gbx_scan_i64(multi, mrow, nrows, st, ws));
    GBX_TRY(gbx_scan_i64(mcnt, mterm, nrows, st, ws));
    int64_t ns = 0, nm = 0, nt = 0;
    GBX_TRY(gbx_read_i64(sidx + nrows, &ns, st));
    GBX_TRY(gbx_read_i64(mrow + nrows, &nm, st));
    GBX_TRY(gbx_read_i64(mterm + nrows, &nt, st));
    if (ns == 0) return GBX_SUCCESS;
    GBX_TRY(req->mem.get(gs, ns + 4)); GBX_TRY(req->mem.get(gd, ns + 4));   // padding for the scatter form
    GBX_TRY(req->mem.get(row_ptr2, nm + 1)); GBX_TRY(req->mem.get(row_out2, nm)); GBX_TRY(req->mem.get(terms2, nt + 2));
    row_split_kernel<<<grid_of(nrows), SETUP_T, 0, st>>>(row_ptr, row_out, terms, nrows, req->elem_size, sidx, mrow,
                                                         mterm, *gs, *gd, *row_ptr2, *row_out2, *terms2, bad);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaMemcpyAsync(*row_ptr2 + nm, &nt, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    int hb = 0;
    GBX_CUDA_TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hb) return GBX_SUCCESS;
    *nsingle = ns;
    *nmulti = nm;
    *nmterms = nt;
    *ok = 1;
    return GBX_SUCCESS;
}

__global__ void check_flat2_kernel(const int32_t *gs, const int32_t *gd, int64_t n, int64_t s, int64_t src_bytes,
                                   int64_t src2_bytes, int64_t dst_bytes, int *err) {
    FOR_EACH(v, n) {
        const uint32_t x = (uint32_t)gs[v];
        const int64_t el = (int64_t)(x & ~GBX_FLAT_SRC2);
        const int64_t lim = (x & GBX_FLAT_SRC2) ? src2_bytes : src_bytes;
        if ((el + 1) * s > lim || gd[v] < 0 || ((int64_t)gd[v] + 1) * s > dst_bytes) set_err(err, GBX_ERR_INTERNAL);
    }
}

// Reorders a two-index copy by its source index (ascending read addresses; bit 31, the
// second buffer, sorts after the first).  Same pairs, same bytes.
__global__ void pair_to_sort_kernel(const int32_t *gs, const int32_t *gd, int64_t n, uint64_t *k, int64_t *v) {
    FOR_EACH(i, n) {
        k[i] = (uint64_t)(uint32_t)gs[i];
        v[i] = gd[i];
    }
}
__global__ void pair_from_sort_kernel(const uint64_t *k, const int64_t *v, int64_t n, int32_t *gs, int32_t *gd) {
    FOR_EACH(i, n) {
        gs[i] = (int32_t)(uint32_t)k[i];
        gd[i] = (int32_t)v[i];
    }
}

int gbx_sort_pairs_by_source(gbx_request_s *req, int32_t *gs, int32_t *gd, int64_t n) {
    cudaStream_t st = req->stream;
    DevPool ws;
    uint64_t *k, *ka;
    int64_t *v, *va;
    GBX_TRY(ws.get(&k, n)); GBX_TRY(ws.get(&ka, n)); GBX_TRY(ws.get(&v, n)); GBX_TRY(ws.get(&va, n));
    pair_to_sort_kernel<<<grid_of(n), SETUP_T, 0, st>>>(gs, gd, n, k, v);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_sort_pairs(&k, &v, ka, va, n, 32, st, ws));
    pair_from_sort_kernel<<<grid_of(n), SETUP_T, 0, st>>>(k, v, n, gs, gd);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return GBX_SUCCESS;
}
