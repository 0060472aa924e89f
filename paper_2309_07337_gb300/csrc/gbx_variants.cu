// gbx_variants.cu -- the other neighbourhood collectives and the dense all-to-all-v, as
// persistent requests on the same engine.
//
// MPI Advance offers its optimised persistent neighbourhood collectives (section 2.2) and
// its all-to-all-v (section 2.1, Listing 2) as drop-in replacements of the MPI calls.  Here
// each of these is the neighbourhood all-to-all-v with counts and displacements derived on
// the device from the graph and the call's arguments, following the MPI standard:
//   neighbor_alltoall:  out-edge j of r sends `count` elements from element j*count;
//                       in-edge i of d receives `count` elements at element i*count;
//   neighbor_allgather: every out-edge of r sends elements [0, count) of r's region;
//                       in-edge i of d receives `count` elements at element i*count;
//   neighbor_allgatherv: every out-edge of r sends elements [0, sendcount[r]);
//                       in-edges receive at the caller's recvcounts / rdispls;
//   alltoallv:          the complete graph (every rank lists every rank, itself included,
//                       in rank order), so the P x P count and displacement matrices are
//                       the per-edge arrays.
#include "gbx_internal.cuh"

#define VT 256
#define FOR_ALL(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static unsigned vgrid(int64_t n) {
    int64_t g = ceil_div(n > 0 ? n : 1, VT);
    return (unsigned)(g > 65535ll * 32 ? 65535ll * 32 : g);
}

// mode 0: alltoall, 1: allgather, 2: allgatherv (per-rank send counts)
// A derived displacement beyond the int32 range of the all-to-all-v arguments is refused
// (GBX_ERR_UNSUPPORTED) on both sides, before any buffer is checked.
__global__ void fill_out_kernel(const int *owner, const int *ptr, int64_t E, int mode, int count,
                                const int *rank_count, int *sendcounts, int *sdispls, int *err) {
    FOR_ALL(e, E) {
        const int r = owner[e];
        const int64_t j = e - ptr[r];
        const int64_t disp = mode == 0 ? j * (int64_t)count : 0;
        if (disp > 0x7fffffffll) atomicMin(err, GBX_ERR_UNSUPPORTED);
        sendcounts[e] = mode == 2 ? rank_count[r] : count;
        sdispls[e] = disp > 0x7fffffffll ? 0 : (int)disp;
    }
}

__global__ void fill_in_kernel(const int *owner, const int *ptr, int64_t E, int count, int *recvcounts,
                               int *rdispls, int *err) {
    FOR_ALL(i, E) {
        const int64_t k = i - ptr[owner[i]];
        const int64_t disp = k * (int64_t)count;
        if (disp > 0x7fffffffll) atomicMin(err, GBX_ERR_UNSUPPORTED);
        recvcounts[i] = count;
        rdispls[i] = disp > 0x7fffffffll ? 0 : (int)disp;
    }
}

static int derived_init(gbx_graph_t graph, int mode, int count, const int *rank_count, const void *sendbuf,
                        int64_t sendbuf_bytes, const int64_t *send_base, void *recvbuf, int64_t recvbuf_bytes,
                        const int64_t *recv_base, const int *recvcounts_in, const int *rdispls_in, int64_t elem_size,
                        int dtype, const char *info, void *stream, gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!graph || (mode != 2 && count < 0) || (mode == 2 && !rank_count)) return GBX_ERR_ARG;
    if (mode == 2 && graph->E > 0 && (!recvcounts_in || !rdispls_in)) return GBX_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t E = graph->E;
    DevPool ws;
    int *sc, *sd, *rc, *rd, *err;
    GBX_TRY(ws.get(&sc, E)); GBX_TRY(ws.get(&sd, E)); GBX_TRY(ws.get(&rc, E)); GBX_TRY(ws.get(&rd, E));
    GBX_TRY(ws.get(&err, 1));
    GBX_CUDA_TRY(cudaMemsetAsync(err, 0x7f, sizeof(int), st));
    if (E > 0) {
        fill_out_kernel<<<vgrid(E), VT, 0, st>>>(graph->out_owner, graph->out_ptr, E, mode, count, rank_count, sc, sd,
                                                 err);
        if (mode != 2) fill_in_kernel<<<vgrid(E), VT, 0, st>>>(graph->in_owner, graph->in_ptr, E, count, rc, rd, err);
        GBX_CUDA_TRY(cudaGetLastError());
    }
    int rc_err = gbx_read_err(err, st);
    if (rc_err == 0x7f7f7f7f) rc_err = GBX_SUCCESS;
    if (rc_err) return rc_err;
    return gbx_neighbor_alltoallv_init(sendbuf, sendbuf_bytes, send_base, sc, sd, nullptr, nullptr, recvbuf,
                                       recvbuf_bytes, recv_base, mode == 2 ? recvcounts_in : rc,
                                       mode == 2 ? rdispls_in : rd, nullptr, elem_size, dtype, nullptr, nullptr, graph,
                                       info, stream, request);
}

extern "C" int gbx_neighbor_alltoall_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                          void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base, int count,
                                          int64_t elem_size, int dtype, gbx_graph_t graph, const char *info,
                                          void *stream, gbx_request_t *request) {
    return derived_init(graph, 0, count, nullptr, sendbuf, sendbuf_bytes, send_base, recvbuf, recvbuf_bytes,
                        recv_base, nullptr, nullptr, elem_size, dtype, info, stream, request);
}

extern "C" int gbx_neighbor_allgather_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                           void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base, int count,
                                           int64_t elem_size, int dtype, gbx_graph_t graph, const char *info,
                                           void *stream, gbx_request_t *request) {
    return derived_init(graph, 1, count, nullptr, sendbuf, sendbuf_bytes, send_base, recvbuf, recvbuf_bytes,
                        recv_base, nullptr, nullptr, elem_size, dtype, info, stream, request);
}

extern "C" int gbx_neighbor_allgatherv_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                            const int *sendcount, void *recvbuf, int64_t recvbuf_bytes,
                                            const int64_t *recv_base, const int *recvcounts, const int *rdispls,
                                            int64_t elem_size, int dtype, gbx_graph_t graph, const char *info,
                                            void *stream, gbx_request_t *request) {
    return derived_init(graph, 2, 0, sendcount, sendbuf, sendbuf_bytes, send_base, recvbuf, recvbuf_bytes,
                        recv_base, recvcounts, rdispls, elem_size, dtype, info, stream, request);
}

// ------------------------------------------------------------ dense alltoallv
__global__ void complete_graph_kernel(int P, int *ptr, int *ranks) {
    const int64_t E = (int64_t)P * P;
    FOR_ALL(i, E) ranks[i] = (int)(i % P);
    FOR_ALL(r, (int64_t)P + 1) ptr[r] = (int)(r * P);
}

extern "C" int gbx_alltoallv_init(gbx_comm_t comm, const void *sendbuf, int64_t sendbuf_bytes,
                                  const int64_t *send_base, const int *sendcounts, const int *sdispls, void *recvbuf,
                                  int64_t recvbuf_bytes, const int64_t *recv_base, const int *recvcounts,
                                  const int *rdispls, int64_t elem_size, int dtype, const char *info, void *stream,
                                  gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!comm) return GBX_ERR_ARG;
    const int64_t P = comm->P;
    if (P * P > 0x7fffffffll) return GBX_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    DevPool ws;
    int *ptr, *ranks;
    GBX_TRY(ws.get(&ptr, P + 1));
    GBX_TRY(ws.get(&ranks, P * P));
    complete_graph_kernel<<<vgrid(P * P), VT, 0, st>>>((int)P, ptr, ranks);
    GBX_CUDA_TRY(cudaGetLastError());
    gbx_graph_t g = nullptr;
    GBX_TRY(gbx_dist_graph_create_adjacent(comm, P * P, ptr, ranks, nullptr, P * P, ptr, ranks, nullptr, nullptr, 0,
                                           stream, &g));
    int rc = gbx_neighbor_alltoallv_init(sendbuf, sendbuf_bytes, send_base, sendcounts, sdispls, nullptr, nullptr,
                                         recvbuf, recvbuf_bytes, recv_base, recvcounts, rdispls, nullptr, elem_size,
                                         dtype, nullptr, nullptr, g, info, stream, request);
    if (rc != GBX_SUCCESS) {
        gbx_graph_free(&g);
        return rc;
    }
    (*request)->owned_graph = g;   // freed with the request
    return GBX_SUCCESS;
}
