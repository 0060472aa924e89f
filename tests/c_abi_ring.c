/* A plain C caller of the library (no Python): a ring of P = 8 ranks, 4 per node, where
 * rank r sends K doubles to rank (r + 1) % P from the send-list elements 2k + 1 of its
 * region; both forms must deliver exactly those values, and the backward must put each
 * received gradient back on the element it came from.  Exit status 0 = every check passed;
 * anything else names the failing check on stderr.  Built and run by
 * tests/test_gpu_c_abi.py against include/gbx.h and libgbx.so. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gbx.h"

#define P 8
#define PPN 4
#define K 3          /* elements per message */
#define NE 8         /* elements per rank region */

#define CHECK(cond, what)                                  \
    do {                                                   \
        if (!(cond)) {                                     \
            fprintf(stderr, "c_abi_ring: %s\n", what);     \
            return 1;                                      \
        }                                                  \
    } while (0)
#define GBX(call) CHECK((call) == GBX_SUCCESS, #call)
#define CU(call) CHECK((call) == cudaSuccess, #call)

static void *dev_copy(const void *h, size_t n) {
    void *d = NULL;
    if (cudaMalloc(&d, n ? n : 1) != cudaSuccess) return NULL;
    if (n && cudaMemcpy(d, h, n, cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
    return d;
}

static int run(const char *info, int *d_in_ptr, int *d_src, int *d_out_ptr, int *d_dst) {
    int cnt[P], sdisp[P], rdisp[P], idx[P * K];
    int64_t send_base[P], recv_base[P], slot_ptr[P + 1];
    double send[P * NE], recv[P * K], grad_recv[P * K], grad_send[P * NE];
    for (int r = 0; r < P; r++) {
        cnt[r] = K;
        sdisp[r] = 0;
        rdisp[r] = 0;
        send_base[r] = (int64_t)r * NE * 8;
        recv_base[r] = (int64_t)r * K * 8;
        for (int k = 0; k < K; k++) idx[r * K + k] = 2 * k + 1;
    }
    for (int r = 0; r <= P; r++) slot_ptr[r] = (int64_t)r * K;
    for (int i = 0; i < P * NE; i++) send[i] = 1000.0 + i;
    for (int i = 0; i < P * K; i++) grad_recv[i] = 0.5 * (i + 1);
    memset(recv, 0, sizeof recv);
    memset(grad_send, 0, sizeof grad_send);

    void *d_send = dev_copy(send, sizeof send), *d_recv = dev_copy(recv, sizeof recv);
    void *d_cnt = dev_copy(cnt, sizeof cnt), *d_sdisp = dev_copy(sdisp, sizeof sdisp);
    void *d_rdisp = dev_copy(rdisp, sizeof rdisp), *d_idx = dev_copy(idx, sizeof idx);
    void *d_sb = dev_copy(send_base, sizeof send_base), *d_rb = dev_copy(recv_base, sizeof recv_base);
    void *d_sp = dev_copy(slot_ptr, sizeof slot_ptr);
    void *d_gr = dev_copy(grad_recv, sizeof grad_recv), *d_gs = dev_copy(grad_send, sizeof grad_send);
    CHECK(d_send && d_recv && d_cnt && d_sdisp && d_rdisp && d_idx && d_sb && d_rb && d_sp && d_gr && d_gs,
          "device buffers");

    gbx_comm_t comm = NULL;
    gbx_graph_t graph = NULL;
    gbx_request_t req = NULL, bwd = NULL;
    GBX(gbx_comm_create(P, PPN, &comm));
    GBX(gbx_dist_graph_create_adjacent(comm, P, d_in_ptr, d_src, NULL, P, d_out_ptr, d_dst, NULL, NULL, 0, NULL,
                                       &graph));
    GBX(gbx_neighbor_alltoallv_init(d_send, sizeof send, d_sb, d_cnt, d_sdisp, d_sp, d_idx, d_recv, sizeof recv,
                                    d_rb, d_cnt, d_rdisp, NULL, 8, GBX_F64, NULL, NULL, graph, info, NULL, &req));
    for (int rep = 0; rep < 2; rep++) {
        GBX(gbx_start(req));
        GBX(gbx_wait(req));
        CU(cudaMemcpy(recv, d_recv, sizeof recv, cudaMemcpyDeviceToHost));
        for (int d = 0; d < P; d++) {
            const int r = (d + P - 1) % P;   /* the sender into d */
            for (int k = 0; k < K; k++)
                CHECK(recv[d * K + k] == send[r * NE + 2 * k + 1], "forward value");
        }
    }
    CHECK(gbx_start(req) == GBX_SUCCESS && gbx_start(req) == GBX_ERR_ACTIVE, "second start while active");
    GBX(gbx_wait(req));
    GBX(gbx_backward_init(req, d_gr, d_gs, 0, info, NULL, &bwd));
    GBX(gbx_start(bwd));
    GBX(gbx_wait(bwd));
    CU(cudaMemcpy(grad_send, d_gs, sizeof grad_send, cudaMemcpyDeviceToHost));
    for (int r = 0; r < P; r++) {
        const int d = (r + 1) % P;   /* the receiver of r's message */
        for (int j = 0; j < NE; j++) {
            const double want = (j % 2 == 1 && j / 2 < K) ? grad_recv[d * K + j / 2] : 0.0;
            CHECK(grad_send[r * NE + j] == want, "backward value");
        }
    }
    GBX(gbx_request_free(&bwd));
    GBX(gbx_request_free(&req));
    GBX(gbx_graph_free(&graph));
    GBX(gbx_comm_free(&comm));
    CHECK(req == NULL && graph == NULL && comm == NULL, "free clears the handles");
    void *bufs[] = {d_send, d_recv, d_cnt, d_sdisp, d_rdisp, d_idx, d_sb, d_rb, d_sp, d_gr, d_gs};
    for (size_t i = 0; i < sizeof bufs / sizeof bufs[0]; i++) cudaFree(bufs[i]);
    return 0;
}

int main(void) {
    int in_ptr[P + 1], out_ptr[P + 1], src[P], dst[P];
    for (int r = 0; r <= P; r++) in_ptr[r] = out_ptr[r] = r;
    for (int r = 0; r < P; r++) {
        src[r] = (r + P - 1) % P;   /* rank r receives from r - 1 */
        dst[r] = (r + 1) % P;       /* and sends to r + 1 */
    }
    int *d_in_ptr = (int *)dev_copy(in_ptr, sizeof in_ptr), *d_out_ptr = (int *)dev_copy(out_ptr, sizeof out_ptr);
    int *d_src = (int *)dev_copy(src, sizeof src), *d_dst = (int *)dev_copy(dst, sizeof dst);
    CHECK(d_in_ptr && d_out_ptr && d_src && d_dst, "graph arrays");
    CHECK(run("algorithm=standard", d_in_ptr, d_src, d_out_ptr, d_dst) == 0, "standard form");
    CHECK(run("algorithm=locality", d_in_ptr, d_src, d_out_ptr, d_dst) == 0, "locality form");
    CHECK(run("algorithm=locality;graph=0;autotune=0", d_in_ptr, d_src, d_out_ptr, d_dst) == 0, "eager locality");
    printf("c_abi_ring ok\n");
    return 0;
}
