// gbx_partition.cu -- device-side setup of the persistent partitioned exchange.
//
// Partitioned communication (MPI Advance section 2.3) lets the parts of a send buffer that
// are ready move before the rest exists.  Here the send buffer is cut into byte ranges
// (partitions); every element of a standard-form forward program is keyed by the partition
// its source lies in and by the receive partition it lands in, the elements are stably
// sorted by send partition (receive order kept inside each), and each partition's elements
// are cut into receive-contiguous runs of one source rank -- the segment + source-index form
// of the standard exchange, so every partition gets an ordinary copy program.  A bitmap
// records which send partitions feed each receive partition.  Errors go to a device word
// with atomicMin; nothing moves on error.
#include <algorithm>
#include <cstring>

#include "gbx_internal.cuh"

#define PT 256
#define P_EACH(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static unsigned pgrid(int64_t n) {
    int64_t g = ceil_div(n > 0 ? n : 1, PT);
    return (unsigned)(g > 65535ll * 32 ? 65535ll * 32 : g);
}

namespace {

struct PArgs {
    const Seg *segs;
    const int64_t *segv0;
    const int *seg_src;
    const int32_t *srcel;
    const int64_t *send_base;
    const int64_t *pp, *rp;   // partition boundaries (npart + 1, nrpart + 1)
    int64_t nseg, V, s;
    int npart, nrpart, words;
};

// largest i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x)
template <typename T>
__device__ __forceinline__ int64_t p_last_le(const T *a, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)a[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void p_elem_kernel(PArgs a, uint64_t *key, int64_t *val, int64_t *sa_out, int64_t *da_out, int *r_out,
                              unsigned long long *cnt, uint32_t *feed, int *err) {
    P_EACH(v, a.V) {
        const int64_t q = p_last_le(a.segv0, a.nseg, v);
        const int r = a.seg_src[q];
        const int64_t sa = a.send_base[r] + (int64_t)a.srcel[v] * a.s;
        const int64_t da = a.segs[q].dst_off + (v - a.segv0[q]) * a.s;
        const int64_t k = p_last_le(a.pp, a.npart, sa);
        const int64_t j = p_last_le(a.rp, a.nrpart, da);
        if (sa + a.s > a.pp[k + 1] || da + a.s > a.rp[j + 1]) atomicMin(err, GBX_ERR_ARG);
        key[v] = (uint64_t)k;
        val[v] = v;
        sa_out[v] = sa;
        da_out[v] = da;
        r_out[v] = r;
        atomicAdd(cnt + k, 1ull);
        atomicOr(feed + j * a.words + (k >> 5), 1u << (k & 31));
    }
}

// segment starts: a new partition or source rank, or a receive address that does not
// continue the previous element's
__global__ void p_flag_kernel(const uint64_t *key, const int64_t *ord, const int64_t *da, const int *rr, int64_t V,
                              int64_t s, int64_t *flag) {
    P_EACH(m, V) {
        int64_t f = 1;
        if (m > 0) {
            const int64_t x = ord[m], y = ord[m - 1];
            f = key[m] != key[m - 1] || rr[x] != rr[y] || da[x] != da[y] + s;
        }
        flag[m] = f;
    }
}

__global__ void p_seg_kernel(PArgs a, const uint64_t *key, const int64_t *ord, const int64_t *da, const int *rr,
                             const int64_t *flag, const int64_t *segid, const int64_t *elem_off, Seg *segs,
                             int32_t *idx, unsigned long long *segcnt) {
    P_EACH(m, a.V) {
        const int64_t x = ord[m];
        const int64_t k = (int64_t)key[m];
        idx[m] = a.srcel[x];
        if (flag[m]) {
            const int64_t rel = m - elem_off[k];
            Seg sg;
            sg.v0 = rel;
            sg.dst_off = da[x];
            sg.src_off = a.send_base[rr[x]];
            sg.idx_off = rel;
            segs[segid[m]] = sg;
            atomicAdd(segcnt + k, 1ull);
        }
    }
}

}  // namespace

int gbx_setup_partitions(gbx_request_s *parent, const gbx_request_s *f, int npart, const int64_t *part_ptr,
                         int nrpart, const int64_t *rpart_ptr, PartPlan *plan) {
    cudaStream_t st = parent->stream;
    const int64_t V = f->V, s = f->elem_size;
    const int words = (npart + 31) / 32;
    DevPool ws;
    int *err;
    int64_t *d_pp, *d_rp;
    unsigned long long *cnt, *segcnt;
    uint32_t *feed;
    GBX_TRY(ws.get(&err, 1));
    GBX_TRY(ws.get(&d_pp, npart + 1));
    GBX_TRY(ws.get(&d_rp, nrpart + 1));
    GBX_TRY(ws.get(&cnt, npart));
    GBX_TRY(ws.get(&segcnt, npart));
    GBX_TRY(ws.get(&feed, (int64_t)nrpart * words));
    GBX_CUDA_TRY(cudaMemcpyAsync(d_pp, part_ptr, sizeof(int64_t) * (npart + 1), cudaMemcpyHostToDevice, st));
    GBX_CUDA_TRY(cudaMemcpyAsync(d_rp, rpart_ptr, sizeof(int64_t) * (nrpart + 1), cudaMemcpyHostToDevice, st));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    GBX_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * npart, st));
    GBX_CUDA_TRY(cudaMemsetAsync(segcnt, 0, sizeof(unsigned long long) * npart, st));
    GBX_CUDA_TRY(cudaMemsetAsync(feed, 0, sizeof(uint32_t) * nrpart * words, st));
    plan->elem_off.assign(npart + 1, 0);
    plan->seg_off.assign(npart + 1, 0);
    plan->feed.assign((size_t)nrpart * words, 0u);
    if (V == 0) return GBX_SUCCESS;

    PArgs a;
    a.segs = f->segs_std; a.segv0 = f->segv0; a.seg_src = f->seg_src_rank; a.srcel = f->srcel;
    a.send_base = f->send_base_copy; a.pp = d_pp; a.rp = d_rp;
    a.nseg = f->nseg; a.V = V; a.s = s; a.npart = npart; a.nrpart = nrpart; a.words = words;
    uint64_t *keyA, *keyB;
    int64_t *valA, *valB, *sa, *da, *flag, *segid, *d_elem_off;
    int *rr;
    GBX_TRY(ws.get(&keyA, V)); GBX_TRY(ws.get(&keyB, V));
    GBX_TRY(ws.get(&valA, V)); GBX_TRY(ws.get(&valB, V));
    GBX_TRY(ws.get(&sa, V)); GBX_TRY(ws.get(&da, V)); GBX_TRY(ws.get(&rr, V));
    p_elem_kernel<<<pgrid(V), PT, 0, st>>>(a, keyA, valA, sa, da, rr, cnt, feed, err);
    GBX_CUDA_TRY(cudaGetLastError());
    int rc = gbx_read_err(err, st);
    if (rc != 0x7f7f7f7f) return rc;
    std::vector<unsigned long long> h(npart);
    GBX_CUDA_TRY(cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * npart, cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaMemcpyAsync(plan->feed.data(), feed, sizeof(uint32_t) * nrpart * words, cudaMemcpyDeviceToHost,
                                 st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < npart; k++) plan->elem_off[k + 1] = plan->elem_off[k] + (int64_t)h[k];
    GBX_TRY(ws.get(&d_elem_off, npart + 1));
    GBX_CUDA_TRY(cudaMemcpyAsync(d_elem_off, plan->elem_off.data(), sizeof(int64_t) * (npart + 1),
                                 cudaMemcpyHostToDevice, st));
    // elements by send partition, receive order kept inside each
    uint64_t *key = keyA;
    int64_t *val = valA;
    GBX_TRY(gbx_sort_pairs(&key, &val, keyB, valB, V, std::max(1, bitlen_u64((uint64_t)npart)), st, ws));
    GBX_TRY(ws.get(&flag, V));
    GBX_TRY(ws.get(&segid, V + 1));
    p_flag_kernel<<<pgrid(V), PT, 0, st>>>(key, val, da, rr, V, s, flag);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(flag, segid, V, st, ws));
    int64_t nseg = 0;
    GBX_TRY(gbx_read_i64(segid + V, &nseg, st));
    GBX_TRY(parent->mem.get(&plan->segs, nseg));
    GBX_TRY(parent->mem.get(&plan->idx, V));
    p_seg_kernel<<<pgrid(V), PT, 0, st>>>(a, key, val, da, rr, flag, segid, d_elem_off, plan->segs, plan->idx,
                                         segcnt);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_CUDA_TRY(cudaMemcpyAsync(h.data(), segcnt, sizeof(unsigned long long) * npart, cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < npart; k++) plan->seg_off[k + 1] = plan->seg_off[k] + (int64_t)h[k];
    if (plan->seg_off[npart] != nseg) return GBX_ERR_INTERNAL;
    return GBX_SUCCESS;
}
