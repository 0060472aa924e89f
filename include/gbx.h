/*
 * gbx.h -- C ABI of a GB300-native persistent neighbourhood all-to-all-v over an
 * emulated distributed-graph communicator whose P ranks keep all their buffers in
 * one GPU's memory.
 *
 * The operation is the one optimised by MPI Advance ("MPI Advance: Open-Source
 * Message Passing Optimizations", arXiv 2309.07337):
 *   - section 2.2, Listing 4: MPIX_Dist_graph_create_adjacent, then
 *     MPIX_Neighbor_alltoallv_init, MPIX_Start, MPIX_Wait; all setup is paid once at
 *     init (section 2.2, first paragraph);
 *   - section 2.2, last paragraph: an optional unique global index per value sent and
 *     received lets the locality-aware form send each value once per pair of nodes;
 *   - section 1: locality-aware aggregation (one message per node pair).
 * The meaning of the exchange is the MPI standard's MPI_Neighbor_alltoallv, which the
 * paper calls (section 2.2, Listing 3) but does not restate.
 *
 * Conventions for every call
 *   - Every function returns GBX_SUCCESS (0) or one of the GBX_ERR_* codes below;
 *     gbx_error_string() gives its text.  On error no handle is returned and no
 *     library memory is left allocated.
 *   - The P emulated ranks live in one process.  Each per-rank MPI argument becomes a
 *     CSR over ranks: in-edge arrays are indexed by the in-list CSR (in_ptr), out-edge
 *     arrays by the out-list CSR (out_ptr).
 *   - Unless stated otherwise, array arguments are DEVICE pointers (setup runs on the
 *     GPU) and are only read during the call; the library keeps its own copies of
 *     whatever it needs, so the caller may free them when the call returns.
 *   - Data buffers (send, receive, gradients) are owned by the caller, bound to the
 *     request at init and used by every start; they must stay valid until the request
 *     is freed (MPI persistent semantics) or re-bound.  They are device memory, or
 *     pinned host memory the GPU can address (cudaHostAlloc / cudaHostRegister): the
 *     kernels then read and write those buffers in place over the host link, so only
 *     the bytes the exchange touches cross it.  The bulk-copy forms (info bulk=) are
 *     not used on host buffers; re-binding an op tuned to one of them to host memory
 *     returns GBX_ERR_UNSUPPORTED.
 *   - Handles are opaque and owned by the library; *_free releases them and sets the
 *     handle to NULL.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Nothing here changes device settings.  The only host-pinned memory the library
 *     allocates is one 64-byte status word per request (mapped, written by its kernels
 *     only when a bounded device wait gives up).
 */
#ifndef GBX_H
#define GBX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (the CPU oracle uses the same numbers) ---- */
#define GBX_SUCCESS          0
#define GBX_ERR_ARG          1   /* NULL / negative / inconsistent argument, not a CSR  */
#define GBX_ERR_RANK         2   /* neighbour rank outside [0, P)                        */
#define GBX_ERR_TRUNCATE     3   /* unmatched edge, or paired counts differ (MPI_ERR_TRUNCATE) */
#define GBX_ERR_INDEX        4   /* displacement, slot or element index out of range     */
#define GBX_ERR_DUP          5   /* one global index carried by different bytes into one
                                    node pair; found at init only with info check_dup=1
                                    (the library otherwise never reads payload at init)    */
#define GBX_ERR_GIDX         6   /* a receive global index differs from the matched send index */
#define GBX_ERR_ACTIVE       7   /* start on a request already started                  */
#define GBX_ERR_TIMEOUT      8   /* wait gave up after the request's timeout; the request
                                    stays active and may be waited on again               */
#define GBX_ERR_CUDA         9   /* a CUDA call failed                                   */
#define GBX_ERR_NOMEM       10   /* device allocation failed                             */
#define GBX_ERR_UNSUPPORTED 11   /* valid request the library does not implement         */
#define GBX_ERR_INTERNAL    12   /* a move program built at init failed the library's own
                                    device-side validation (a library bug); nothing ran    */
#define GBX_ERR_OVERLAP     13   /* two receive blocks write the same bytes              */
#define GBX_ERR_LIMIT       14   /* beyond the fixed capacity of gbx_neighbor_alltoallv_noalloc */
#define GBX_ERR_STATE       15   /* call not allowed in the request's current state (partitioned:
                                    pready before start or twice in one epoch, a wait or an
                                    arrival wait before the partitions it needs were marked) */
#define GBX_ERR_DEVICE_WAIT 16   /* the exchange finished on the GPU but incomplete: a bounded
                                    wait of one of its kernels on its own copies gave up (or a
                                    move piece failed the kernel's own check); the receive
                                    buffer is partly written.  Reported once by gbx_wait /
                                    gbx_test / gbx_waitall; the request is then inactive and
                                    may be started again */

/* payload types: only the backward (which adds) needs to know them */
#define GBX_BYTES 0
#define GBX_F32   1
#define GBX_F64   2

/* algorithms */
#define GBX_ALG_STANDARD 0   /* pack by send index list, block copy, unpack          */
#define GBX_ALG_LOCALITY 1   /* direct intra-node copy + three-step aggregation      */

typedef struct gbx_comm_s *gbx_comm_t;
typedef struct gbx_graph_s *gbx_graph_t;
typedef struct gbx_request_s *gbx_request_t;

/* What a request does per start; filled by gbx_request_get_info. */
typedef struct {
    int kind;               /* 0 forward exchange, 1 backward (reverse) exchange, 2 partitioned */
    int algorithm;          /* GBX_ALG_*                                              */
    int levels;             /* dependent kernel phases per start (1 or 3)             */
    int launches;           /* kernels per start                                      */
    int use_graph;          /* 1 if start replays a captured CUDA graph               */
    int vec_bytes;          /* vector width of the dominant move kernel               */
    int block;              /* threads per block of the dominant move kernel          */
    int unroll;             /* chunks per thread per tile of the dominant kernel      */
    int64_t elem_size;
    int64_t V;              /* elements moved by the standard form                    */
    int64_t E;              /* matched edges (messages), zero-count ones included     */
    int64_t E_nonzero;      /* edges that carry data                                  */
    int64_t V_direct;       /* locality form: elements moved inside a node            */
    int64_t V_inter;        /* elements whose sender and receiver are on different nodes */
    int64_t U;              /* locality form: distinct inter-node values (step 1 = step 2 volume) */
    int64_t node_pairs;     /* locality form: node pairs with traffic (= step 2 messages) */
    int64_t msgs_inter;     /* standard form: inter-node messages                     */
    int64_t msgs_intra;     /* standard form: intra-node messages                     */
    int64_t msgs_step1;     /* locality form: ranks sending to a different send leader */
    int64_t msgs_step3;     /* locality form: receive leaders sending to another rank  */
    int64_t rows;           /* backward: distinct source elements written             */
    int64_t terms;          /* backward: additive terms read                          */
    int64_t user_bytes;     /* 2*V*elem_size: bytes a user sees moved                 */
    int64_t algo_bytes;     /* bytes the method must read and write per start,
                               index and descriptor reads included                    */
    int64_t device_bytes;   /* device memory the request owns                         */
    int64_t copy_forms;     /* bit f set when some copy runs in form f: 0 segments,
                               1 gather, 3 two-index, 5/7 pipelined 1/3, 8 bulk pieces,
                               9 source windows scattered, 10/11 stream forms of 1/3;
                               bit 12: a fold runs in its stream form (fixed at init by
                               the tuner) */
} gbx_request_info_t;

const char *gbx_error_string(int code);
int gbx_version(void);

/* Emulated communicator of P ranks, ranks_per_node consecutive ranks per node
 * (node(r) = r / ranks_per_node; the last node may be smaller).  Stands in for
 * MPIX_Comm_init (section 2.1, Listing 2).  Host-only; no device memory. */
int gbx_comm_create(int P, int ranks_per_node, gbx_comm_t *comm);
int gbx_comm_free(gbx_comm_t *comm);

/* Distributed graph (MPI_Dist_graph_create_adjacent, section 2.2 Listings 3-4) over
 * all P ranks at once.
 *   in_ptr[P+1], sources[n_in_edges]:   rank d's in-neighbours are
 *                                       sources[in_ptr[d] .. in_ptr[d+1]-1];
 *   out_ptr[P+1], destinations[n_out_edges]: likewise for out-neighbours.
 *   sourceweights / destweights: accepted (may be NULL) and ignored, as is `reorder`
 *                                (no rank reordering).
 *   info: reserved, may be NULL.
 * Device kernels validate the CSRs (GBX_ERR_ARG), the ranks (GBX_ERR_RANK) and match
 * every out-edge r->d with an in-edge of d under the MPI multigraph rule (the t-th
 * listing of d by r pairs with the t-th listing of r by d); an edge without a partner
 * gives GBX_ERR_TRUNCATE.  Blocks on `stream` once to read the result.
 * The graph keeps a pointer to `comm`, which must outlive it. */
int gbx_dist_graph_create_adjacent(gbx_comm_t comm,
                                   int64_t n_in_edges, const int *in_ptr, const int *sources,
                                   const int *sourceweights,
                                   int64_t n_out_edges, const int *out_ptr,
                                   const int *destinations, const int *destweights,
                                   const char *info, int reorder, void *stream,
                                   gbx_graph_t *graph);
int gbx_graph_free(gbx_graph_t *graph);

/* Persistent neighbourhood all-to-all-v (MPIX_Neighbor_alltoallv_init, section 2.2
 * Listing 4).  For every out-edge e of rank r to d, paired with in-edge i of d:
 *     recv[d][rdispls[i] + k] = send[r][elem_r(sdispls[e] + k)],  0 <= k < sendcounts[e]
 * where element j of rank r's send region starts at byte send_base[r] + j*elem_size of
 * sendbuf, element j of d's receive region at byte recv_base[d] + j*elem_size of
 * recvbuf, and elem_r(q) = send_idx[send_slot_ptr[r] + q] when send_idx is given (the
 * pack-by-send-index-list step), else q (a user-packed send buffer).
 *
 *   sendbuf, sendbuf_bytes     send buffer of all ranks (device, or pinned host memory; a
 *                              pageable host pointer gives GBX_ERR_ARG) and its size in bytes
 *   send_base[P]               byte offset of each rank's send region (int64)
 *   sendcounts, sdispls        per out-edge, in elements (int32, >= 0)
 *   send_slot_ptr[P+1]         CSR of send slots; required with send_idx or global_sidx,
 *                              then sdispls[e] + sendcounts[e] <= slots of r; else NULL
 *   send_idx                   per send slot, element index in the rank's region; or NULL
 *   recvbuf, recvbuf_bytes     receive buffer of all ranks (same rules) and its size
 *   recv_base[P]               byte offset of each rank's receive region
 *   recvcounts, rdispls        per in-edge, in elements; recvcounts must equal the paired
 *                              sendcounts (else GBX_ERR_TRUNCATE)
 *   recv_slot_ptr[P+1]         CSR of receive slots (bounds rdispls); required with
 *                              global_ridx; else NULL
 *   elem_size                  bytes per element (any positive size)
 *   dtype                      GBX_BYTES, GBX_F32 or GBX_F64; only the backward uses it
 *   global_sidx, global_ridx   unique global index of every send / receive slot (int64;
 *                              section 2.2, last paragraph), or NULL.  The locality form
 *                              aggregates by it; without it a value is named by its
 *                              source element (its byte offset in the send buffer), so an
 *                              element sent to several ranks of one remote node crosses
 *                              that node pair once.  global_ridx is optional and, when
 *                              given, must equal the paired send index (GBX_ERR_GIDX).
 *                              The same global index sent by two ranks of one node to
 *                              the same remote node must carry identical bytes: it is
 *                              sent once, from the first such sender in out-edge order.
 *   graph, info, stream, request
 *   info: "key=value;..." with
 *       algorithm=standard|locality|auto   (default standard; auto times both and keeps
 *                                          the faster)
 *       graph=0|1          capture the start sequence in a CUDA graph (default 1)
 *       autotune=0|1       time candidate kernel shapes at init (default 1)
 *       vec=V block=B      force the move kernel's vector width / block size
 *       min_run=N          gathered runs of >= N consecutive source elements are copied as
 *                          contiguous blocks (default 4; 0 keeps every element gathered)
 *       flat=0|1           force / forbid the flat form of a copy (one contiguous destination
 *                          run, one source index per element, no segment search); by
 *                          default the autotuner picks it where it applies
 *       piece=N            run copies in ascending source order, in pieces of <= N elements
 *                          (default 0: receive order)
 *       timeout_ms=T       limit of gbx_wait (default 60000)
 *       bulk=0|1|2         offer the bulk form (contiguous pieces moved through shared memory
 *                          by the bulk-copy engine) to the autotuner where every block is
 *                          contiguous and 16-byte aligned (default 1; 2 forces it there).
 *                          In a backward the same key offers (1) or forces (2) the scatter
 *                          form of the single-term rows: source windows read by the
 *                          bulk-copy engine, scattered to their destinations by the threads
 *       stream=0|1|2       offer the stream form of the flat copies (the per-element index
 *                          arrays copied into shared memory ahead of the payload loads by the
 *                          bulk-copy engine) to the autotuner (default 1; 0 leaves it out, 2
 *                          forces it where it applies: index arrays the library built, vectors
 *                          of at least 4 bytes)
 *       form=F             the autotuner times only copy form F (a bit number of copy_forms
 *                          below) in every copy that offers it, the others as usual (default
 *                          -1); for reproducing one program shape, e.g. under a profiler
 *       max_ctas=N         at most N thread blocks in any launch (default 0: no cap), leaving
 *                          the rest of the GPU to other requests' kernels on other streams;
 *                          every move kernel covers its work with any grid
 *       check_dup=0|1      locality form: at init, compare the bytes of every element that
 *                          shares a (node pair, global index) value with the value's
 *                          representative in the send buffer as bound then (default 0)
 *       wait_limit=N       polls (N >= 0, default 4194304) of each main wait of the kernels
 *                          that wait on their own asynchronous copies (the bulk-copy and
 *                          scatter forms) before the wait gives up and the start reports
 *                          GBX_ERR_DEVICE_WAIT; waits that drain copies already in flight
 *                          keep the default.  In a batch the first request's limit applies
 * Errors: GBX_ERR_ARG, _TRUNCATE, _INDEX, _GIDX, _OVERLAP (receive blocks must not
 * overlap), _DUP (with check_dup=1), _NOMEM, _CUDA.  Validation and map building run as device kernels; the
 * call blocks on `stream` to read their status.  The autotuner's trial launches write
 * the bound receive buffer (with the correct result for the send data present then).
 * Element bytes are copied exactly; no value is converted. */
int gbx_neighbor_alltoallv_init(const void *sendbuf, int64_t sendbuf_bytes,
                                const int64_t *send_base, const int *sendcounts,
                                const int *sdispls, const int64_t *send_slot_ptr,
                                const int *send_idx,
                                void *recvbuf, int64_t recvbuf_bytes,
                                const int64_t *recv_base, const int *recvcounts,
                                const int *rdispls, const int64_t *recv_slot_ptr,
                                int64_t elem_size, int dtype,
                                const int64_t *global_sidx, const int64_t *global_ridx,
                                gbx_graph_t graph, const char *info, void *stream,
                                gbx_request_t *request);

/* The other neighbourhood collectives, persistent, on the same engine (MPI Advance offers
 * its persistent neighbourhood collectives as drop-in replacements of the MPI calls,
 * section 2.2; their meaning is the MPI standard's).  Each derives per-edge counts and
 * displacements on the device from the graph, then behaves as gbx_neighbor_alltoallv_init
 * with user-packed buffers and no global indices (info keys apply as there; with
 * algorithm=locality a value is named by its source element, so the allgathers send each
 * element once per remote node).  `count` / `sendcount` are in elements.
 *   neighbor_alltoall:   rank r sends `count` elements to its j-th out-neighbour from element
 *                        j*count of its send region; rank d receives `count` elements from its
 *                        i-th in-neighbour at element i*count of its receive region.
 *   neighbor_allgather:  rank r sends its elements [0, count) to every out-neighbour; rank d
 *                        receives them from in-neighbour i at element i*count.
 *   neighbor_allgatherv: rank r sends its elements [0, sendcount[r]) to every out-neighbour
 *                        (sendcount: device int[P]); rank d receives recvcounts[i] elements from
 *                        in-neighbour i at element rdispls[i] (recvcounts must equal the
 *                        sender's count, else GBX_ERR_TRUNCATE).
 * Errors as gbx_neighbor_alltoallv_init, plus GBX_ERR_UNSUPPORTED when a derived displacement
 * exceeds the int32 range. */
int gbx_neighbor_alltoall_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                               void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                               int count, int64_t elem_size, int dtype, gbx_graph_t graph,
                               const char *info, void *stream, gbx_request_t *request);
int gbx_neighbor_allgather_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                                int count, int64_t elem_size, int dtype, gbx_graph_t graph,
                                const char *info, void *stream, gbx_request_t *request);
int gbx_neighbor_allgatherv_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                 const int *sendcount, void *recvbuf, int64_t recvbuf_bytes,
                                 const int64_t *recv_base, const int *recvcounts, const int *rdispls,
                                 int64_t elem_size, int dtype, gbx_graph_t graph,
                                 const char *info, void *stream, gbx_request_t *request);

/* Reads and clears the process-wide status word of the move kernels, the aggregate of every
 * request's own word: 1 when a bounded wait of the bulk or scatter kernel gave up since the
 * last call (the launch then left its pieces unfinished), 2 when one of their pieces failed
 * its in-kernel check and was skipped, else 0.  Each request also has its own word, which
 * gbx_wait / gbx_test read (GBX_ERR_DEVICE_WAIT).  No counterpart in the paper. */
int gbx_device_status(int *status);

/* Persistent partitioned exchange (section 2.3: partitioned communication lets marked
 * portions of a buffer move before the whole message is complete -- early-bird transfer --
 * and lets the receiver use completed portions early).  Built on a standard-form forward
 * request `forward` (from gbx_neighbor_alltoallv_init, the derived collectives or
 * gbx_neighbor_alltoallw_init; the locality form gives GBX_ERR_UNSUPPORTED), which must
 * outlive it and keeps working on its own.
 *   part_ptr[npart+1]    HOST byte boundaries of the send partitions over the forward's
 *                        send buffer: part_ptr[0] = 0, non-decreasing, part_ptr[npart] =
 *                        sendbuf_bytes; element bytes the exchange reads may not straddle a
 *                        boundary (GBX_ERR_ARG otherwise).  1 <= npart <= 1024.
 *   rpart_ptr[nrpart+1]  HOST byte boundaries of the receive partitions over the receive
 *                        buffer, same rules.  1 <= nrpart <= 1024.
 * Each send partition's elements (those whose source lies in it) get their own move
 * program, built, validated, tuned and captured at init.  Use, per epoch:
 *   gbx_start(req)                       opens an epoch (no data moves yet);
 *   gbx_pready(req, p, stream)           partition p is ready: its moves are enqueued on
 *                                        `stream` (NULL = the request's stream), ordered
 *                                        after the producer's work already on that stream;
 *   gbx_parrived(req, j, &flag)          flag = 1 once every value of receive partition j
 *                                        has landed (host query, no blocking);
 *   gbx_parrived_stream(req, j, stream)  `stream` waits (on the device) until receive
 *                                        partition j has landed; every send partition
 *                                        feeding j must have been marked (GBX_ERR_STATE);
 *   gbx_wait / gbx_test / gbx_wait_stream   complete the epoch; every partition must have
 *                                        been marked (GBX_ERR_STATE otherwise; the epoch
 *                                        stays open).
 * Nothing waits on the device for a flag: readiness is stream order, so a partition
 * produced by a kernel on stream A moves right after it when marked on A.  gbx_startall
 * and gbx_start_host do not take partitioned requests (GBX_ERR_UNSUPPORTED);
 * gbx_request_bind rebinds every partition's program. */
int gbx_partitioned_init(gbx_request_t forward, int npart, const int64_t *part_ptr, int nrpart,
                         const int64_t *rpart_ptr, const char *info, void *stream,
                         gbx_request_t *request);
int gbx_pready(gbx_request_t request, int partition, void *stream);
int gbx_parrived(gbx_request_t request, int rpartition, int *flag);
int gbx_parrived_stream(gbx_request_t request, int rpartition, void *stream);

/* Datatype of gbx_neighbor_alltoallw_init: a block of `blocklen` bytes repeated over three
 * strided levels, innermost first (count[0] blocks stride[0] bytes apart form a row,
 * count[1] rows stride[1] apart a plane, count[2] planes stride[2] apart an item), and
 * consecutive items `extent` bytes apart.  This is an MPI hvector nested up to three times
 * and resized to `extent`, with lower bound 0 (MPI_Type_create_subarray of a 3D block is one
 * such type).  Size of one item = blocklen * count[0] * count[1] * count[2] bytes; its type
 * map lists item by item, level 2, level 1, level 0, then the block's bytes in order.
 * Every field must be >= 0 and the size at most 2^31 bytes (else GBX_ERR_ARG); an unused
 * level has count 1. */
typedef struct {
    int64_t blocklen;
    int64_t count[3];
    int64_t stride[3];
    int64_t extent;
} gbx_datatype_t;

/* Persistent neighbourhood all-to-all-w (MPI_Neighbor_alltoallw: the neighbourhood
 * collectives of section 2.2 with one datatype per edge; meaning of the MPI standard).
 * Out-edge j of rank r sends sendcounts[j] items of datatype types[sendtypes[j]], starting
 * sdispls[j] BYTES into r's send region (send_base[r]); in-edge i of rank d receives
 * recvcounts[i] items of types[recvtypes[i]] starting rdispls[i] bytes into d's receive
 * region.  Matched edges (the t-th listing rule of gbx_dist_graph_create_adjacent) must
 * carry the same number of bytes; the k-th byte of the send type map lands on the k-th byte
 * of the receive type map.  Receive bytes no message covers are untouched.
 *   sendcounts, sendtypes: device int[E] aligned with the destinations; sdispls: device
 *   int64[E];  recvcounts, recvtypes: device int[E] aligned with the sources; rdispls:
 *   device int64[E];  send_base, recv_base: device int64[P];  types: HOST array of
 *   `ntypes` datatypes, copied at init;  dtype: payload type for a backward request
 *   (GBX_BYTES / F32 / F64).
 * The exchange runs as the standard form (info algorithm=standard or absent; other values
 * give GBX_ERR_UNSUPPORTED) over units of u bytes, u the largest power of two <= 16
 * dividing every block length, stride and extent of the table and every base and
 * displacement.  gbx_backward_init accepts the request when u is a multiple of the payload
 * size: each payload element then receives the sum of the gradients at the receive
 * elements it was copied to, in (destination rank, receive address) order.
 * Errors, the smallest code winning: GBX_ERR_ARG (null argument, bad datatype or datatype
 * index), GBX_ERR_RANK / GBX_ERR_TRUNCATE (unmatched edges, unequal byte counts, negative
 * counts), GBX_ERR_INDEX (negative base or displacement, a byte outside its buffer),
 * GBX_ERR_OVERLAP (a receive byte written twice), GBX_ERR_UNSUPPORTED (more than 2^31
 * units in a rank's send region or in total, or P and the receive buffer too large to key
 * in 64 bits).  Nothing is launched on error. */
int gbx_neighbor_alltoallw_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                const int *sendcounts, const int64_t *sdispls, const int *sendtypes,
                                void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                                const int *recvcounts, const int64_t *rdispls, const int *recvtypes,
                                const gbx_datatype_t *types, int ntypes, int dtype, gbx_graph_t graph,
                                const char *info, void *stream, gbx_request_t *request);

/* Persistent all-to-all-v over the emulated communicator (MPIX_Alltoallv, section 2.1,
 * Listing 2): rank r sends sendcounts[r*P + d] elements from element sdispls[r*P + d] of its
 * send region to rank d, which stores them at element rdispls[d*P + r] of its receive region
 * (recvcounts[d*P + r] must match).  All four arrays are device int[P*P], row-major by rank.
 * The library builds the complete graph (every rank, itself included, in rank order) and
 * frees it with the request.  Other arguments as gbx_neighbor_alltoallv_init; with
 * info algorithm=locality the dense traffic takes the locality-aware form (one aggregate
 * per node pair, values named by their source elements). */
int gbx_alltoallv_init(gbx_comm_t comm, const void *sendbuf, int64_t sendbuf_bytes,
                       const int64_t *send_base, const int *sendcounts, const int *sdispls,
                       void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                       const int *recvcounts, const int *rdispls, int64_t elem_size, int dtype,
                       const char *info, void *stream, gbx_request_t *request);

/* Reverse exchange of a forward request: the transpose of its 0/1 map (the exchange is
 * linear), so that a halo exchange can be differentiated.  grad_recv has the forward
 * receive buffer's layout, grad_send the forward send buffer's.  Every source element
 * read by at least one receive slot gets the sum of those slots' gradients:
 *   standard forward: one left-to-right sum over the slots ordered by (destination rank,
 *     receive position);
 *   locality forward: the reverse of the three steps -- per distinct inter-node value
 *     the sum over its slots in (rank, position) order, carried back across the node
 *     pair, then per source element its groups folded in ascending destination node
 *     (its own node's group = its direct slots in (rank, position) order).
 * accumulate=0 stores the sum, accumulate=1 adds it to the existing value; elements no
 * slot reads are never written.  Init's autotuner may write grad_send (with the correct
 * sums for the gradients present then) when accumulate=0; with accumulate=1 it never
 * launches, so grad_send is untouched until the first start.  Adds are IEEE round-to-nearest in the payload type
 * (dtype of the forward must be GBX_F32 or GBX_F64, elem_size a multiple of it); the
 * order is fixed, so results are bitwise reproducible.  Buffers and base offsets must be
 * aligned to the payload type (GBX_ERR_UNSUPPORTED otherwise).  The forward request must
 * outlive the backward one.  info: graph=, autotune=, timeout_ms=, vec=, block=, bulk= as
 * above; single_split=0 keeps rows with a single term in the summing kernel (by default,
 * without accumulate, such rows are plain copies and run as one two-index gather-scatter);
 * split_order=auto|source|dest orders that copy's pairs by source or by destination (auto,
 * the default: by source where the scatter form can run, that is 16-byte elements and
 * alignment with bulk forms allowed, so the autotuner may pick it; else by destination);
 * bulk=2 forces the scatter form where it applies. */
int gbx_backward_init(gbx_request_t forward, const void *grad_recv, void *grad_send,
                      int accumulate, const char *info, void *stream,
                      gbx_request_t *request);

/* MPIX_Start (section 2.2, Listing 4): enqueues one exchange on the request's stream
 * (one CUDA graph launch, or eager kernel launches when graph=0).  GBX_ERR_ACTIVE if
 * the request was started and not yet completed by wait/test. */
int gbx_start(gbx_request_t request);

/* MPIX_Wait (section 2.2, Listing 4): blocks the host until the started exchange has
 * finished on the GPU, polling with a limit of timeout_ms (the calling thread polls
 * without sleeping for the first 20 ms, then sleeps 20 us between polls); returns
 * GBX_ERR_TIMEOUT (request still active) when the limit passes.  An inactive request returns at once.
 * When the exchange finished but one of its kernels gave up a bounded wait (see
 * GBX_ERR_DEVICE_WAIT and info wait_limit), returns GBX_ERR_DEVICE_WAIT and clears the
 * request's status word; the request is inactive either way.  On an inactive request it
 * reports (and clears) a status word left set by an exchange completed with
 * gbx_wait_stream, once that exchange's kernels have finished. */
int gbx_wait(gbx_request_t request);

/* Non-blocking completion check: *flag = 1 and the request becomes inactive if done; the
 * return code reports a device wait that gave up as gbx_wait does. */
int gbx_test(gbx_request_t request, int *flag);

/* Completes a started request without blocking the host: `stream` waits for it on the
 * GPU and the request becomes inactive (stream-ordered use, e.g. autograd).  It cannot
 * read the request's status word (the kernels have not finished yet): a device wait that
 * gave up stays recorded and is reported by the request's next gbx_wait or gbx_test. */
int gbx_wait_stream(gbx_request_t request, void *stream);

/* Starts `count` inactive requests as one batch: all their move phases run as fused
 * multi-pattern kernels (one launch per dependent phase, every pattern's tiles in the
 * same grid), replayed from one CUDA graph built and cached on the first call for this
 * exact request list (that first call allocates and blocks once).  The batch runs on
 * requests[0]'s stream; each request completes through gbx_wait/gbx_waitall.  The
 * requests must write disjoint memory. */
int gbx_startall(int count, gbx_request_t *requests);
int gbx_waitall(int count, gbx_request_t *requests);

/* Re-binds the data buffers of an inactive request without redoing setup: `src` is the
 * new send buffer (grad_recv for a backward request), `dst` the new receive buffer
 * (grad_send); NULL keeps the old one.  The new buffers must have the sizes of the old
 * ones; one aligned below the vector width a move program of the request was tuned to
 * gives GBX_ERR_ARG (the old binding stays).  Batches of gbx_startall that hold their own
 * wider copies of the request's programs move them to the new buffers, and a batch whose
 * copies the new buffers no longer align is rebuilt at its next gbx_startall.  The new
 * descriptors are uploaded on the request's stream; a request that belongs to a cached
 * batch (which may run on another request's stream) synchronises that stream first. */
int gbx_request_bind(gbx_request_t request, const void *src, void *dst);

/* One exchange on HOST buffers: copies host_src (the whole bound source buffer, pinned
 * host memory recommended) to the bound device source buffer, starts the exchange, and
 * copies the bound destination buffer back to host_dst, all on the request's stream;
 * then waits as gbx_wait does. */
int gbx_start_host(gbx_request_t request, const void *host_src, void *host_dst);

/* The same on HOST buffers without blocking: enqueues (1) the copy of host_src to the
 * bound device source buffer on the request's own upload stream, after the work already
 * queued on the request's stream (the earlier exchanges that read that buffer); (2) the
 * exchange on the request's stream, after that copy; (3) the copy of the bound destination
 * buffer to host_dst on the request's own download stream, after the exchange.  host_src =
 * NULL skips (1) (the device source is used as it is: e.g. a second request over the same
 * source, started after the first on the same stream); host_dst = NULL skips (3).  The
 * request completes (gbx_wait, gbx_test, gbx_wait_stream) once (3), else (2), is done;
 * its next exchange, from any start call, is ordered after (3).  Successive calls on two
 * requests whose buffers differ overlap one's upload with the other's download: the two
 * copy directions use separate copy engines.  host_src and host_dst must stay valid and
 * unchanged until completion; pinned memory makes the copies asynchronous.  Errors:
 * GBX_ERR_ARG, _ACTIVE, _UNSUPPORTED (partitioned requests), _CUDA. */
int gbx_start_host_async(gbx_request_t request, const void *host_src, void *host_dst);

int gbx_request_get_info(gbx_request_t request, gbx_request_info_t *info);

/* Largest edge count gbx_neighbor_alltoallv_noalloc accepts (in-edges and out-edges). */
#define GBX_NOALLOC_MAX_EDGES (1 << 18)

/* One standard neighbourhood all-to-all-v, executed now, that allocates no memory.
 * The paper has no counterpart of this call; it exists for callers that cannot call
 * cudaMalloc: code running under a fixed memory budget whose free memory another
 * allocator already owns (a framework's caching allocator), latency-critical paths
 * that cannot afford cudaMalloc's implicit device-wide synchronisation, and plug-ins or
 * callbacks that are not allowed to touch the allocator.  It does no persistent setup
 * and returns no handle: every call matches, validates and moves in one go.
 *   Meaning: that of gbx_neighbor_alltoallv_init with send_idx, the slot CSRs and the
 *   global indices all NULL (a user-packed send buffer): for every in-edge i of rank d
 *   from r, paired under the multigraph rule with out-edge e of r,
 *     recv bytes [recv_base[d] + rdispls[i]*s, +recvcounts[i]*s) =
 *     send bytes [send_base[r] + sdispls[e]*s, +sendcounts[e]*s).
 *   Arguments: as gbx_dist_graph_create_adjacent and gbx_neighbor_alltoallv_init.  The
 *   index and count arrays (in_ptr, sources, out_ptr, destinations, send_base,
 *   sendcounts, sdispls, recv_base, recvcounts, rdispls) are device memory; sendbuf and
 *   recvbuf are device memory or pinned host memory the GPU can address (read and written
 *   in place); a pageable host pointer gives GBX_ERR_ARG before any device work.  All of
 *   them stay owned by the caller.
 *   Scratch: the per-edge tables live in one file-scope device array sized for
 *   GBX_NOALLOC_MAX_EDGES edges (about 6 MB).  Edge counts above the limit return
 *   GBX_ERR_LIMIT before any device work.  CUDA loads a library's device code lazily by
 *   default, so the first call on a device loads the part of the library that holds the
 *   array, which reserves its 6 MB of device memory, and looks the array's device address
 *   up (cudaGetSymbolAddress) with that device current; make that first call while the
 *   device still has that memory free and before any stream capture.  From then on the
 *   device holds the array until the process exits and no call allocates anything.  All
 *   calls on a device share the array and a call overwrites what the previous one left
 *   there, so calls that may overlap on the GPU (different streams, other host threads)
 *   race and must be serialised by the caller.
 *   Errors: GBX_ERR_ARG, _RANK, _TRUNCATE, _INDEX, _LIMIT, _CUDA as in the persistent
 *   path; overlapping receive blocks are not detected (MPI makes them erroneous).
 *   The call enqueues its kernels on `stream` and blocks until they finish, then returns
 *   the status; nothing is written to the receive buffer unless every check passed. */
int gbx_neighbor_alltoallv_noalloc(int P, int64_t n_in_edges, const int *in_ptr, const int *sources,
                                   int64_t n_out_edges, const int *out_ptr, const int *destinations,
                                   const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                   const int *sendcounts, const int *sdispls,
                                   void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                                   const int *recvcounts, const int *rdispls,
                                   int64_t elem_size, void *stream);

/* MPI_Request_free: waits for an active request, then releases its device memory and
 * any cached batch that contains it. */
int gbx_request_free(gbx_request_t *request);

#ifdef __cplusplus
}
#endif

#endif /* GBX_H */
