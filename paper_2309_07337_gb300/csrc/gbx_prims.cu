// gbx_prims.cu -- device building blocks of the setup phase: an exclusive scan and a
// stable LSD radix sort, written for this library (no CUB / Thrust).  They run once
// per persistent request init, never on the exchange path.
#include <cstdio>
#include <cstring>

#include "gbx_internal.cuh"

void gbx_note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    if (getenv("GBX_DEBUG"))
        fprintf(stderr, "gbx: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
}

int DevPool::alloc(void **p, size_t n) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GBX_ERR_NOMEM;
    }
    ptrs.push_back(*p);
    bytes += (int64_t)n;
    return GBX_SUCCESS;
}

void DevPool::release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
}

// --------------------------------------------------------------------------- scan
// 512 threads x 8 consecutive items per block.
#define SCAN_T 512
#define SCAN_I 8
#define SCAN_TILE (SCAN_T * SCAN_I)

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total, int64_t *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem[32 + lane] = w;  // inclusive warp prefix
    }
    __syncthreads();
    int64_t warp_excl = warp ? smem[32 + warp - 1] : 0;
    *total = smem[32 + (blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_excl + x - v;
}

__global__ void scan_reduce_kernel(const int64_t *in, int64_t n, int64_t *partial) {
    __shared__ int64_t smem[64];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++)
        if (base + i < n) s += in[base + i];
    int64_t tot;
    block_excl_scan(s, &tot, smem);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// out[i] = offset[block] + exclusive prefix inside the block; out[n] = total (last block)
__global__ void scan_apply_kernel(const int64_t *in, int64_t n, const int64_t *offset, int64_t *out) {
    __shared__ int64_t smem[64];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t v[SCAN_I];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t pre = block_excl_scan(s, &tot, smem) + (offset ? offset[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = pre;
}

int gbx_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st, DevPool &ws) {
    if (n <= 0) {
        GBX_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
        return GBX_SUCCESS;
    }
    int64_t nb = ceil_div(n, SCAN_TILE);
    if (nb == 1) {
        scan_apply_kernel<<<1, SCAN_T, 0, st>>>(in, n, nullptr, out);
        GBX_CUDA_TRY(cudaGetLastError());
        return GBX_SUCCESS;
    }
    int64_t *partial, *poff;
    GBX_TRY(ws.get(&partial, nb));
    GBX_TRY(ws.get(&poff, nb + 1));
    scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, partial);
    GBX_CUDA_TRY(cudaGetLastError());
    GBX_TRY(gbx_scan_i64(partial, poff, nb, st, ws));
    scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, poff, out);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_SUCCESS;
}

// --------------------------------------------------------------------- radix sort
// 256 threads; each block owns RS_SUB sub-tiles of 256 consecutive items.
#define RS_T 256
#define RS_SUB 16
#define RS_TILE (RS_T * RS_SUB)

__global__ void radix_hist_kernel(const uint64_t *keys, int64_t n, int shift, int64_t nb,
                                  int64_t *counts) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int s = 0; s < RS_SUB; s++) {
        int64_t i = base + (int64_t)s * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t *keys, const int64_t *vals, int64_t n, int shift,
                                     int64_t nb, const int64_t *offsets, uint64_t *okeys,
                                     int64_t *ovals) {
    __shared__ int64_t run[256];
    __shared__ unsigned int wc[RS_T / 32][256];
    __shared__ unsigned int tot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    run[tid] = offsets[(int64_t)tid * nb + blockIdx.x];
    for (int w = 0; w < RS_T / 32; w++) wc[w][tid] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int s = 0; s < RS_SUB; s++) {
        int64_t i = base + (int64_t)s * RS_T + tid;
        bool valid = i < n;
        uint64_t k = valid ? keys[i] : 0;
        int64_t v = valid ? vals[i] : 0;
        unsigned int digit = valid ? (unsigned int)((k >> shift) & 0xff) : 256u + lane;
        unsigned int peers = __match_any_sync(0xffffffffu, digit);
        unsigned int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wc[warp][digit] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, and the sub-tile total
            unsigned int acc = 0;
            for (int w = 0; w < RS_T / 32; w++) {
                unsigned int c = wc[w][tid];
                wc[w][tid] = acc;
                acc += c;
            }
            tot[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = run[digit] + wc[warp][digit] + rank;
            okeys[pos] = k;
            ovals[pos] = v;
        }
        __syncthreads();
        run[tid] += tot[tid];
        for (int w = 0; w < RS_T / 32; w++) wc[w][tid] = 0;
        __syncthreads();
    }
}

int gbx_sort_pairs(uint64_t **keys, int64_t **vals, uint64_t *keys_alt, int64_t *vals_alt,
                   int64_t n, int bits, cudaStream_t st, DevPool &ws) {
    if (n <= 1 || bits <= 0) return GBX_SUCCESS;
    int64_t nb = ceil_div(n, RS_TILE);
    int64_t *counts, *offsets;
    GBX_TRY(ws.get(&counts, 256 * nb));
    GBX_TRY(ws.get(&offsets, 256 * nb + 1));
    uint64_t *k0 = *keys, *k1 = keys_alt;
    int64_t *v0 = *vals, *v1 = vals_alt;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_kernel<<<(unsigned)nb, RS_T, 0, st>>>(k0, n, shift, nb, counts);
        GBX_CUDA_TRY(cudaGetLastError());
        GBX_TRY(gbx_scan_i64(counts, offsets, 256 * nb, st, ws));
        radix_scatter_kernel<<<(unsigned)nb, RS_T, 0, st>>>(k0, v0, n, shift, nb, offsets, k1, v1);
        GBX_CUDA_TRY(cudaGetLastError());
        uint64_t *tk = k0; k0 = k1; k1 = tk;
        int64_t *tv = v0; v0 = v1; v1 = tv;
    }
    *keys = k0;
    *vals = v0;
    return GBX_SUCCESS;
}

// ----------------------------------------------------------------------- helpers
__global__ void fill_i64_kernel(int64_t *p, int64_t v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
__global__ void iota_i64_kernel(int64_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = i;
}

static unsigned grid_for(int64_t n) {
    int64_t g = ceil_div(n, 256);
    return (unsigned)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

int gbx_fill_i64(int64_t *p, int64_t v, int64_t n, cudaStream_t st) {
    if (n <= 0) return GBX_SUCCESS;
    fill_i64_kernel<<<grid_for(n), 256, 0, st>>>(p, v, n);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_SUCCESS;
}

int gbx_iota_i64(int64_t *p, int64_t n, cudaStream_t st) {
    if (n <= 0) return GBX_SUCCESS;
    iota_i64_kernel<<<grid_for(n), 256, 0, st>>>(p, n);
    GBX_CUDA_TRY(cudaGetLastError());
    return GBX_SUCCESS;
}

int gbx_read_i64(const int64_t *d, int64_t *h, cudaStream_t st) {
    GBX_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return GBX_SUCCESS;
}

int gbx_read_err(int *d_err, cudaStream_t st) {
    int h = GBX_ERR_NONE;
    GBX_CUDA_TRY(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return h == GBX_ERR_NONE ? GBX_SUCCESS : h;
}
