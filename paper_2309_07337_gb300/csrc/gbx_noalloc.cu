// gbx_noalloc.cu -- a one-shot standard neighbourhood all-to-all-v that allocates no
// memory, for callers that cannot call cudaMalloc (see gbx_neighbor_alltoallv_noalloc in
// include/gbx.h).
//
// The persistent path keeps its per-edge tables in memory it allocates at init.  Here the
// same tables (matched source / destination offsets and the running element count of
// every in-edge) live in one file-scope device array of fixed size, so a call needs no
// allocation at all.  Every call on a device shares that array: a call clears what must
// start at zero (the status word) before using it, and calls whose work overlaps on the
// GPU race on it.
#include <mutex>

#include "gbx_internal.cuh"

#define NA_T 256
#define NA_NONE 0x7f7f7f7f

// Layout of the scratch array (offsets in bytes):
//   [0, 256)                       status word, OR of offsets (vector width), V
//   [256, 256 + 8 (E + 1))          element start of every in-edge (scan output)
//   then 8 E                        byte offset of the matched send block
//   then 8 E                        byte offset of the receive block
static const int64_t NA_HDR = 256;
static const int64_t NA_BYTES = NA_HDR + 8 * (GBX_NOALLOC_MAX_EDGES + 1) + 16 * (int64_t)GBX_NOALLOC_MAX_EDGES;

static __device__ __align__(256) unsigned char gbx_noalloc_scratch[NA_BYTES];

struct NaHeader {
    int err;                 // lowest error code seen (NA_NONE = none)
    int pad;
    unsigned long long orv;  // OR of every base, displacement offset and the element size
    long long V;             // elements to move
};

struct NaView {
    NaHeader *h;
    int64_t *v0;
    int64_t *soff;
    int64_t *doff;
};

__device__ __forceinline__ NaView na_view(unsigned char *base) {
    NaView v;
    v.h = reinterpret_cast<NaHeader *>(base);
    v.v0 = reinterpret_cast<int64_t *>(base + NA_HDR);
    v.soff = v.v0 + (GBX_NOALLOC_MAX_EDGES + 1);
    v.doff = v.soff + GBX_NOALLOC_MAX_EDGES;
    return v;
}

__device__ __forceinline__ void na_err(NaView v, int code) { atomicMin(&v.h->err, code); }

struct NaArgs {
    int P;
    int64_t E, Eo;           // in-edges, out-edges
    const int *in_ptr, *sources, *out_ptr, *dests;
    const int64_t *send_base, *recv_base;
    const int *sendcounts, *sdispls, *recvcounts, *rdispls;
    int64_t s, send_bytes, recv_bytes;
};

// structure: CSRs, ranks and per-rank bases
__global__ void na_check_kernel(unsigned char *scratch, NaArgs a) {
    NaView v = na_view(scratch);
    int64_t n = (a.E > a.Eo) ? a.E : a.Eo;
    if (n < a.P + 1) n = a.P + 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i <= a.P) {
            if (i == 0 && (a.in_ptr[0] != 0 || a.out_ptr[0] != 0)) na_err(v, GBX_ERR_ARG);
            if (i == a.P && ((int64_t)a.in_ptr[a.P] != a.E || (int64_t)a.out_ptr[a.P] != a.Eo)) na_err(v, GBX_ERR_ARG);
            if (i < a.P && (a.in_ptr[i + 1] < a.in_ptr[i] || a.out_ptr[i + 1] < a.out_ptr[i])) na_err(v, GBX_ERR_ARG);
            if (i < a.P && (a.send_base[i] < 0 || a.recv_base[i] < 0)) na_err(v, GBX_ERR_INDEX);
            if (i < a.P) atomicOr(&v.h->orv, (unsigned long long)(a.send_base[i] | a.recv_base[i]));
        }
        if (i < a.E && (a.sources[i] < 0 || a.sources[i] >= a.P)) na_err(v, GBX_ERR_RANK);
        if (i < a.Eo && (a.dests[i] < 0 || a.dests[i] >= a.P)) na_err(v, GBX_ERR_RANK);
    }
}

// largest r in [0, P) with ptr[r] <= e (valid CSR assumed: checked by the previous kernel)
__device__ __forceinline__ int na_owner(const int *ptr, int P, int64_t e) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if ((int64_t)ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// per in-edge i of rank d from r: its t-th listing of r pairs with r's t-th listing of d
__global__ void na_match_kernel(unsigned char *scratch, NaArgs a) {
    NaView v = na_view(scratch);
    if (v.h->err <= GBX_ERR_RANK) return;   // the lists themselves are invalid
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.E; i += (int64_t)gridDim.x * blockDim.x) {
        v.v0[i] = 0;
        const int d = na_owner(a.in_ptr, a.P, i);
        const int r = a.sources[i];
        int64_t t = 0;
        for (int64_t j = a.in_ptr[d]; j < i; j++) t += a.sources[j] == r;
        int64_t e = -1;
        for (int64_t j = a.out_ptr[r]; j < a.out_ptr[r + 1]; j++)
            if (a.dests[j] == d && t-- == 0) { e = j; break; }
        if (e < 0) { na_err(v, GBX_ERR_TRUNCATE); continue; }
        const int64_t cnt = a.recvcounts[i];
        if ((int64_t)a.sendcounts[e] != cnt || cnt < 0) { na_err(v, GBX_ERR_TRUNCATE); continue; }
        const int64_t sd = a.sdispls[e], rd = a.rdispls[i];
        // bounds by division, so that no product can overflow whatever the element size:
        // base + (disp + cnt) * s <= bytes  <=>  disp + cnt <= (bytes - base) / s
        const int64_t sb = a.send_base[r], rb = a.recv_base[d];
        if (sd < 0 || rd < 0 || sb > a.send_bytes || rb > a.recv_bytes || sd + cnt > (a.send_bytes - sb) / a.s ||
            rd + cnt > (a.recv_bytes - rb) / a.s) {
            na_err(v, GBX_ERR_INDEX);
            continue;
        }
        v.v0[i] = cnt;
        v.soff[i] = a.send_base[r] + sd * a.s;
        v.doff[i] = a.recv_base[d] + rd * a.s;
        atomicOr(&v.h->orv, (unsigned long long)(v.soff[i] | v.doff[i]));
    }
}

// exclusive scan of the counts in place (one block; E <= GBX_NOALLOC_MAX_EDGES)
__global__ void na_scan_kernel(unsigned char *scratch, int64_t E) {
    NaView v = na_view(scratch);
    if (v.h->err != NA_NONE) return;
    __shared__ int64_t part[1024];
    const int64_t per = (E + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * per, hi = lo + per < E ? lo + per : E;
    int64_t sum = 0;
    for (int64_t i = lo; i < hi; i++) sum += v.v0[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (unsigned k = 0; k < blockDim.x; k++) { int64_t x = part[k]; part[k] = acc; acc += x; }
        v.h->V = acc;
        v.v0[E] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = lo; i < hi; i++) { int64_t x = v.v0[i]; v.v0[i] = acc; acc += x; }
}

template <int VEC>
__device__ __forceinline__ void na_copy_chunk(const char *src, char *dst) {
    if (VEC == 16) *reinterpret_cast<uint4 *>(dst) = __ldg(reinterpret_cast<const uint4 *>(src));
    else if (VEC == 8) *reinterpret_cast<uint2 *>(dst) = __ldg(reinterpret_cast<const uint2 *>(src));
    else if (VEC == 4) *reinterpret_cast<unsigned *>(dst) = __ldg(reinterpret_cast<const unsigned *>(src));
    else if (VEC == 2) *reinterpret_cast<unsigned short *>(dst) = __ldg(reinterpret_cast<const unsigned short *>(src));
    else *dst = *src;
}

template <int VEC>
__device__ void na_copy(NaView v, const char *src, char *dst, int64_t E, int64_t s) {
    const int64_t cpe = s / VEC;
    const int64_t nchunks = (int64_t)v.h->V * cpe;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t el = c / cpe, j = c - el * cpe;
        int64_t lo = 0, hi = E - 1;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) >> 1;
            if (v.v0[mid] <= el) lo = mid; else hi = mid - 1;
        }
        const int64_t k = el - v.v0[lo];
        na_copy_chunk<VEC>(src + v.soff[lo] + k * s + j * VEC, dst + v.doff[lo] + k * s + j * VEC);
    }
}

__global__ void na_copy_kernel(unsigned char *scratch, const char *src, char *dst, int64_t E, int64_t s,
                               unsigned long long ptr_or) {
    NaView v = na_view(scratch);
    if (v.h->err != NA_NONE || v.h->V == 0) return;   // nothing moves unless every check passed
    const unsigned long long o = v.h->orv | ptr_or | (unsigned long long)s;
    if (!(o & 15)) na_copy<16>(v, src, dst, E, s);
    else if (!(o & 7)) na_copy<8>(v, src, dst, E, s);
    else if (!(o & 3)) na_copy<4>(v, src, dst, E, s);
    else if (!(o & 1)) na_copy<2>(v, src, dst, E, s);
    else na_copy<1>(v, src, dst, E, s);
}

// Device address of the scratch array, looked up once per device with that device current.
static std::mutex g_na_mu;
static unsigned char *g_na_ptr[64];

static int na_scratch(unsigned char **out) {
    int dev = 0;
    GBX_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        GBX_CUDA_TRY(cudaGetSymbolAddress(&p, gbx_noalloc_scratch));
        g_na_ptr[dev] = (unsigned char *)p;
    }
    *out = g_na_ptr[dev];
    return GBX_SUCCESS;
}

extern "C" int gbx_neighbor_alltoallv_noalloc(int P, int64_t n_in_edges, const int *in_ptr, const int *sources,
                                              int64_t n_out_edges, const int *out_ptr, const int *destinations,
                                              const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                              const int *sendcounts, const int *sdispls, void *recvbuf,
                                              int64_t recvbuf_bytes, const int64_t *recv_base, const int *recvcounts,
                                              const int *rdispls, int64_t elem_size, void *stream) {
    if (P <= 0 || n_in_edges < 0 || n_out_edges < 0 || elem_size <= 0 || sendbuf_bytes < 0 || recvbuf_bytes < 0)
        return GBX_ERR_ARG;
    if (!in_ptr || !out_ptr || !send_base || !recv_base) return GBX_ERR_ARG;
    if ((sendbuf_bytes > 0 && !sendbuf) || (recvbuf_bytes > 0 && !recvbuf)) return GBX_ERR_ARG;
    if (n_in_edges > 0 && (!sources || !recvcounts || !rdispls)) return GBX_ERR_ARG;
    if (n_out_edges > 0 && (!destinations || !sendcounts || !sdispls)) return GBX_ERR_ARG;
    if (n_in_edges > GBX_NOALLOC_MAX_EDGES || n_out_edges > GBX_NOALLOC_MAX_EDGES) return GBX_ERR_LIMIT;
    GbxRange range("gbx.noalloc");
    GBX_TRY(gbx_check_data_buf(sendbuf, sendbuf_bytes));
    GBX_TRY(gbx_check_data_buf(recvbuf, recvbuf_bytes));
    unsigned char *scratch = nullptr;
    GBX_TRY(na_scratch(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    // what must start at zero: the status word, the offset OR and the element count
    NaHeader h0;
    memset(&h0, 0, sizeof(h0));
    h0.err = NA_NONE;
    GBX_CUDA_TRY(cudaMemcpyAsync(scratch, &h0, sizeof(h0), cudaMemcpyHostToDevice, st));
    NaArgs a;
    a.P = P; a.E = n_in_edges; a.Eo = n_out_edges; a.in_ptr = in_ptr; a.sources = sources; a.out_ptr = out_ptr; a.dests = destinations;
    a.send_base = send_base; a.recv_base = recv_base; a.sendcounts = sendcounts; a.sdispls = sdispls;
    a.recvcounts = recvcounts; a.rdispls = rdispls; a.s = elem_size; a.send_bytes = sendbuf_bytes;
    a.recv_bytes = recvbuf_bytes;
    // structure first, so that GBX_ERR_ARG / GBX_ERR_RANK take precedence over TRUNCATE
    int err = n_in_edges != n_out_edges ? GBX_ERR_TRUNCATE : GBX_SUCCESS;
    int64_t n = n_in_edges > n_out_edges ? n_in_edges : n_out_edges;
    if (n < P + 1) n = P + 1;
    int64_t g = ceil_div(n, NA_T);
    if (g > 4096) g = 4096;
    na_check_kernel<<<(unsigned)g, NA_T, 0, st>>>(scratch, a);
    GBX_CUDA_TRY(cudaGetLastError());
    if (err == GBX_SUCCESS && a.E > 0) {
        int64_t ge = ceil_div(a.E, NA_T);
        if (ge > 4096) ge = 4096;
        na_match_kernel<<<(unsigned)ge, NA_T, 0, st>>>(scratch, a);
        na_scan_kernel<<<1, 1024, 0, st>>>(scratch, a.E);
        const unsigned long long ptr_or = (unsigned long long)(uintptr_t)sendbuf | (unsigned long long)(uintptr_t)recvbuf;
        na_copy_kernel<<<(unsigned)(gbx_num_sms() * 8), 256, 0, st>>>(scratch, (const char *)sendbuf, (char *)recvbuf,
                                                                      a.E, elem_size, ptr_or);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    NaHeader h;
    GBX_CUDA_TRY(cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.err != NA_NONE && (err == GBX_SUCCESS || h.err < err)) err = h.err;
    return err;
}
