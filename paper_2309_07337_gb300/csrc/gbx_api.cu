// gbx_api.cu -- the C ABI (include/gbx.h): communicator, distributed graph, persistent
// requests (init / start / wait, MPI Advance section 2.2 Listing 4), batched start,
// re-binding, the autotuner and CUDA-graph capture.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>

#include "gbx_internal.cuh"

struct Batch {
    std::vector<gbx_request_s *> members;
    DevPool mem;
    std::vector<LevelLaunch> launches;
    std::vector<HostOp> widened;   // batch-owned copies of ops re-cut to their widest vector
    std::vector<std::pair<gbx_request_s *, size_t>> widened_of;   // (request, op index) of each
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
};

extern "C" const char *gbx_error_string(int code) {
    switch (code) {
        case GBX_SUCCESS: return "success";
        case GBX_ERR_ARG: return "invalid argument";
        case GBX_ERR_RANK: return "neighbour rank out of range";
        case GBX_ERR_TRUNCATE: return "unmatched edge or count mismatch between paired edges";
        case GBX_ERR_INDEX: return "displacement or index out of range";
        case GBX_ERR_DUP: return "one global index carried by different bytes";
        case GBX_ERR_GIDX: return "receive global index differs from the paired send index";
        case GBX_ERR_ACTIVE: return "request already active";
        case GBX_ERR_TIMEOUT: return "wait timed out";
        case GBX_ERR_CUDA: return "CUDA error";
        case GBX_ERR_NOMEM: return "out of device memory";
        case GBX_ERR_UNSUPPORTED: return "unsupported request";
        case GBX_ERR_OVERLAP: return "receive blocks overlap";
        case GBX_ERR_INTERNAL: return "internal error: a generated move program failed validation";
        case GBX_ERR_LIMIT: return "size beyond the fixed scratch of the allocation-free exchange";
        case GBX_ERR_STATE: return "call not allowed in the request's current state";
        case GBX_ERR_DEVICE_WAIT: return "a bounded device wait gave up: the exchange is incomplete";
        default: return "unknown error";
    }
}

extern "C" int gbx_version(void) { return 100; }

extern "C" int gbx_device_status(int *status) {
    if (!status) return GBX_ERR_ARG;
    return gbx_bulk_status_take(status);
}

// ------------------------------------------------------------------------ info
struct Opts {
    int algorithm = GBX_ALG_STANDARD;
    int algorithm_auto = 0;
    int graph = 1, autotune = 1, vec = 0, block = 0, timeout_ms = 60000, min_run = 4, piece = 0, flat = -1;
    int split = 1, split_order = 2;   // 2: source order where the scatter form can run, else dest
    int check_dup = 0, bulk = 1, max_ctas = 0, wait_limit = GBX_WAIT_LIMIT, stream = 1, form = -1;
    bool ok = true;
};

static Opts parse_info(const char *info) {
    Opts o;
    if (!info) return o;
    std::string s(info);
    size_t pos = 0;
    while (pos < s.size()) {
        size_t end = s.find(';', pos);
        if (end == std::string::npos) end = s.size();
        std::string kv = s.substr(pos, end - pos);
        pos = end + 1;
        if (kv.empty()) continue;
        size_t eq = kv.find('=');
        if (eq == std::string::npos) { o.ok = false; continue; }
        std::string k = kv.substr(0, eq), v = kv.substr(eq + 1);
        if (k == "algorithm") {
            if (v == "standard") o.algorithm = GBX_ALG_STANDARD;
            else if (v == "locality") o.algorithm = GBX_ALG_LOCALITY;
            else if (v == "auto") o.algorithm_auto = 1;
            else o.ok = false;
        } else if (k == "graph") o.graph = atoi(v.c_str()) != 0;
        else if (k == "autotune") o.autotune = atoi(v.c_str()) != 0;
        else if (k == "vec") o.vec = atoi(v.c_str());
        else if (k == "block") o.block = atoi(v.c_str());
        else if (k == "timeout_ms") o.timeout_ms = atoi(v.c_str());
        else if (k == "min_run") o.min_run = atoi(v.c_str());
        else if (k == "piece") o.piece = atoi(v.c_str());
        else if (k == "flat") o.flat = atoi(v.c_str()) != 0;
        else if (k == "single_split") o.split = atoi(v.c_str()) != 0;
        else if (k == "split_order") o.split_order = v == "source" ? 1 : v == "dest" ? 0 : v == "auto" ? 2 : -1;
        else if (k == "check_dup") o.check_dup = atoi(v.c_str()) != 0;
        else if (k == "bulk") o.bulk = atoi(v.c_str());
        else if (k == "max_ctas") o.max_ctas = atoi(v.c_str());
        else if (k == "wait_limit") o.wait_limit = atoi(v.c_str());
        else if (k == "stream") o.stream = atoi(v.c_str());
        else if (k == "form") o.form = atoi(v.c_str());
        else o.ok = false;
    }
    if (o.vec && !(o.vec == 1 || o.vec == 2 || o.vec == 4 || o.vec == 8 || o.vec == 16)) o.ok = false;
    if (o.block && !(o.block == 128 || o.block == 256 || o.block == 512 || o.block == 1024)) o.ok = false;
    if (o.timeout_ms <= 0 || o.min_run < 0 || o.piece < 0 || o.split_order < 0) o.ok = false;
    if (o.bulk < 0 || o.bulk > 2 || o.max_ctas < 0 || o.wait_limit < 0 || o.stream < 0 || o.stream > 2) o.ok = false;
    if (o.form < -1 || o.form > 11) o.ok = false;
    return o;
}

// ----------------------------------------------------------------- comm, graph
extern "C" int gbx_comm_create(int P, int ranks_per_node, gbx_comm_t *comm) {
    if (!comm) return GBX_ERR_ARG;
    *comm = nullptr;
    if (P <= 0 || ranks_per_node <= 0) return GBX_ERR_ARG;
    gbx_comm_s *c = new gbx_comm_s;
    c->P = P;
    c->ppn = ranks_per_node;
    c->nnodes = (P + ranks_per_node - 1) / ranks_per_node;
    *comm = c;
    return GBX_SUCCESS;
}

extern "C" int gbx_comm_free(gbx_comm_t *comm) {
    if (!comm) return GBX_ERR_ARG;
    delete *comm;
    *comm = nullptr;
    return GBX_SUCCESS;
}

extern "C" int gbx_dist_graph_create_adjacent(gbx_comm_t comm, int64_t n_in_edges, const int *in_ptr,
                                              const int *sources, const int *sourceweights, int64_t n_out_edges,
                                              const int *out_ptr, const int *destinations, const int *destweights,
                                              const char *info, int reorder, void *stream, gbx_graph_t *graph) {
    (void)sourceweights; (void)destweights; (void)info; (void)reorder;
    GbxRange range("gbx.setup.graph");
    if (!graph) return GBX_ERR_ARG;
    *graph = nullptr;
    if (!comm || n_in_edges < 0 || n_out_edges < 0 || !in_ptr || !out_ptr) return GBX_ERR_ARG;
    if ((n_in_edges > 0 && !sources) || (n_out_edges > 0 && !destinations)) return GBX_ERR_ARG;
    gbx_graph_s *g = new gbx_graph_s();
    g->comm = comm;
    g->P = comm->P;
    g->ppn = comm->ppn;
    g->nnodes = comm->nnodes;
    cudaGetDevice(&g->device);
    int rc = gbx_graph_setup(g, n_in_edges, in_ptr, sources, n_out_edges, out_ptr, destinations,
                             (cudaStream_t)stream);
    if (rc != GBX_SUCCESS) {
        delete g;
        return rc;
    }
    *graph = g;
    return GBX_SUCCESS;
}

extern "C" int gbx_graph_free(gbx_graph_t *graph) {
    if (!graph) return GBX_ERR_ARG;
    delete *graph;
    *graph = nullptr;
    return GBX_SUCCESS;
}

// ------------------------------------------------------------------------- ops
// Host memory the kernels can address (pinned, mapped): buffers there are read and written in
// place over the host link.  The bulk-copy forms are not used on them; the index-driven
// kernels are.
static bool host_mem(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// A data buffer must be memory the GPU can address: device, managed, or pinned / registered
// host memory.  Pageable host memory is refused (GBX_ERR_ARG) rather than faulted on.
int gbx_check_data_buf(const void *p, int64_t bytes) {
    if (!p || bytes <= 0) return GBX_SUCCESS;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return GBX_ERR_ARG;
    }
    return a.type == cudaMemoryTypeUnregistered ? GBX_ERR_ARG : GBX_SUCCESS;
}

static int vec_of_align(uint64_t align) {
    int v = 16;
    while (v > 1 && (align & (uint64_t)(v - 1))) v >>= 1;
    return v;
}

// The stream forms read the flat form's index arrays with the bulk-copy engine, in 16-byte
// pieces that may run up to 3 entries past the end: the arrays must be 16-byte aligned and
// padded by 4 entries (every flat index array the library builds is), and the vector width
// at least 4 bytes.
static int stream_ok_for(const gbx_request_s *req, const int32_t *g, const int32_t *gd, int max_vec) {
    static int prepared = 0;
    if (!req->allow_stream || max_vec < 4 || ((uintptr_t)g & 15) || ((uintptr_t)gd & 15)) return 0;
    if (!prepared) {
        if (gbx_stream_prepare() != GBX_SUCCESS) return 0;
        prepared = 1;
    }
    return 1;
}

int gbx_make_copy_op(gbx_request_s *req, int level, const char *src, int src_role, char *dst, int dst_role,
                     const Seg *segs, int64_t nseg, const int32_t *idx, int64_t idx_len, int64_t nelem,
                     int64_t algo_bytes) {
    if (nelem <= 0) return GBX_SUCCESS;
    if (idx && req->min_run > 0) {
        // contiguous source runs become contiguous segments (same elements, same bytes)
        Seg *split = nullptr;
        int64_t nsplit = 0;
        GBX_TRY(gbx_split_runs(req, segs, nseg, idx, nelem, req->min_run, &split, &nsplit));
        algo_bytes += (nsplit - nseg) * (int64_t)sizeof(Seg);
        segs = split;
        nseg = nsplit;
    }
    if (req->piece > 0) {
        // pieces in ascending source address (same elements, same bytes)
        const int64_t src_bytes = src_role == ROLE_SRC ? req->src_bytes : 2 * req->Ur * req->elem_size;
        Seg *ord = nullptr;
        int64_t nord = 0;
        GBX_TRY(gbx_order_by_source(req, segs, nseg, idx, nelem, src_bytes, req->piece, &ord, &nord));
        algo_bytes += (nord - nseg) * (int64_t)sizeof(Seg);
        segs = ord;
        nseg = nord;
    }
    HostOp op;
    memset(&op, 0, sizeof(op));
    op.kind = 0;
    op.level = level;
    op.units = nelem;
    op.max_vec = vec_of_align(req->align);
    op.min_vec = req->forced_vec ? std::min(req->forced_vec, op.max_vec) : std::max(1, op.max_vec / 2);
    if (req->forced_vec) op.max_vec = op.min_vec;
    op.block = 256;
    op.persistent = 1;
    op.algo_bytes = algo_bytes;
    op.idx_len = idx_len;
    CopyDesc &d = op.cd;
    d.src = src; d.dst = dst; d.segs = segs; d.idx = idx; d.nseg = nseg; d.nelem = nelem;
    d.elem_size = req->elem_size; d.src_role = src_role; d.dst_role = dst_role;
    d.status = req->status_dev; d.wait_limit = req->wait_limit;
    const int64_t max_tiles = ceil_div(nelem * (req->elem_size / op.min_vec), GBX_TILE);
    GBX_TRY(req->mem.get(&op.d_tile_seg, max_tiles + 1));
    GBX_TRY(req->mem.get(&op.d_tile_e0, max_tiles + 1));
    GBX_TRY(req->mem.alloc(&op.d_desc, sizeof(CopyDesc)));
    GBX_TRY(req->mem.get(&op.d_self, 1));
    GBX_TRY(req->mem.get(&op.d_self_prefix, 2));
    d.tile_seg = op.d_tile_seg;
    d.tile_e0 = op.d_tile_e0;
    if (req->allow_flat) {
        GBX_TRY(gbx_make_flat(req, segs, nseg, idx, nelem, &op.d_flat_idx, &op.flat_dst0, &op.flat_ok));
        d.flat_idx = op.d_flat_idx;
        d.dst_flat0 = op.flat_dst0;
        op.algo_bytes_flat = 2 * nelem * req->elem_size + 4 * nelem;
        op.stream_ok = op.flat_ok && stream_ok_for(req, op.d_flat_idx, nullptr, op.max_vec);
    }
    if (req->allow_bulk && !host_mem(src) && !host_mem(dst)) {
        GBX_TRY(gbx_make_bulk(req, segs, nseg, nelem, src_role == ROLE_AGG && dst_role == ROLE_AGG, &op.d_bulk,
                              &op.nbulk, &op.bulk_ok));
        d.bulk = op.d_bulk;
        d.nbulk = op.nbulk;
        op.algo_bytes_bulk = 2 * nelem * req->elem_size + op.nbulk * (int64_t)sizeof(BulkTask);
    }
    op.algo_bytes_seg = op.algo_bytes;
    req->ops.push_back(op);
    return GBX_SUCCESS;
}

int gbx_make_flat_op(gbx_request_s *req, int level, const char *src, int src_role, const char *src2, int src2_role,
                     char *dst, int dst_role, const int32_t *g, int64_t nelem, int64_t dst0) {
    if (nelem <= 0) return GBX_SUCCESS;
    HostOp op;
    memset(&op, 0, sizeof(op));
    op.kind = 0;
    op.level = level;
    op.units = nelem;
    op.max_vec = vec_of_align(req->align);
    op.min_vec = req->forced_vec ? std::min(req->forced_vec, op.max_vec) : std::max(1, op.max_vec / 2);
    if (req->forced_vec) op.max_vec = op.min_vec;
    op.block = 256;
    op.persistent = 1;
    op.flat_ok = 1;
    op.flat_only = 1;
    op.algo_bytes = op.algo_bytes_flat = 2 * nelem * req->elem_size + 4 * nelem;
    op.idx_len = 0;
    op.d_flat_idx = (int32_t *)g;
    op.flat_dst0 = dst0;
    CopyDesc &d = op.cd;
    d.src = src; d.dst = dst; d.segs = nullptr; d.idx = nullptr; d.nseg = 0; d.nelem = nelem;
    d.elem_size = req->elem_size; d.src_role = src_role; d.dst_role = dst_role;
    d.flat = 1; d.flat_idx = g; d.dst_flat0 = dst0; d.src2 = src2; d.src2_role = src2_role;
    d.status = req->status_dev; d.wait_limit = req->wait_limit;
    op.stream_ok = stream_ok_for(req, g, nullptr, op.max_vec);
    const int64_t max_tiles = ceil_div(nelem * (req->elem_size / op.min_vec), GBX_TILE);
    GBX_TRY(req->mem.get(&op.d_tile_e0, max_tiles + 1));
    d.tile_e0 = op.d_tile_e0;
    GBX_TRY(req->mem.alloc(&op.d_desc, sizeof(CopyDesc)));
    GBX_TRY(req->mem.get(&op.d_self, 1));
    GBX_TRY(req->mem.get(&op.d_self_prefix, 2));
    req->ops.push_back(op);
    return GBX_SUCCESS;
}

// Single-term pairs run in source order when asked for, or by default where the scatter form
// (16-byte elements and alignment, bulk forms allowed) can use them.
static bool pairs_in_source_order(const gbx_request_s *req) {
    return req->split_order == 1 ||
           (req->split_order == 2 && req->allow_bulk && (req->elem_size & 15) == 0 && (req->align & 15) == 0);
}

int gbx_make_flat2_op(gbx_request_s *req, int level, const char *src, int src_role, const char *src2, int src2_role,
                      char *dst, int dst_role, const int32_t *gs, const int32_t *gd, int64_t nelem) {
    GBX_TRY(gbx_make_flat_op(req, level, src, src_role, src2, src2_role, dst, dst_role, gs, nelem, 0));
    HostOp &op = req->ops.back();
    op.cd.flat = 3;
    op.cd.flat_didx = gd;
    op.stream_ok = op.stream_ok && stream_ok_for(req, gs, gd, op.max_vec);
    op.algo_bytes = op.algo_bytes_flat = 2 * nelem * req->elem_size + 8 * nelem;
    if (req->allow_bulk && pairs_in_source_order(req) && nelem > 0 && !host_mem(src) && !host_mem(dst)) {
        GBX_TRY(gbx_make_scatter(req, gs, nelem, &op.d_scat, &op.nscat, &op.scat_ok));
        op.cd.scat = op.d_scat;
        op.cd.nscat = op.nscat;
        op.algo_bytes_scat = 2 * nelem * req->elem_size + 8 * nelem + op.nscat * (int64_t)sizeof(ScatterPiece);
    }
    return GBX_SUCCESS;
}

int gbx_make_fold_op(gbx_request_s *req, int level, char *out, int out_role, const char *bufA, int a_role,
                     const char *bufB, int b_role, const int64_t *row_ptr, const int64_t *row_out,
                     const int64_t *terms, int64_t nrows, int64_t nterms, int accumulate) {
    if (nrows <= 0) return GBX_SUCCESS;
    if (!accumulate && !req->no_single_split) {
        // rows with one term are copies: a two-index flat copy op takes them
        int32_t *gs = nullptr, *gd = nullptr;
        int64_t *rp2 = nullptr, *ro2 = nullptr, *t2 = nullptr, ns = 0, nm = 0, nt = 0;
        int ok = 0;
        GBX_TRY(gbx_split_single_rows(req, row_ptr, row_out, terms, nrows, &gs, &gd, &ns, &rp2, &ro2, &t2, &nm, &nt,
                                      &ok));
        if (ok) {
            // source order (also what the scatter form needs); the two-index kernels run
            // equally fast in either order
            if (pairs_in_source_order(req)) GBX_TRY(gbx_sort_pairs_by_source(req, gs, gd, ns));
            GBX_TRY(gbx_make_flat2_op(req, level, bufA, a_role, bufB, b_role, out, out_role, gs, gd, ns));
            if (nm == 0) return GBX_SUCCESS;
            row_ptr = rp2;
            row_out = ro2;
            terms = t2;
            nrows = nm;
            nterms = nt;
        }
    }
    HostOp op;
    memset(&op, 0, sizeof(op));
    op.kind = 1;
    op.level = level;
    op.units = nrows;
    const int dsz = req->dtype == GBX_F64 ? 8 : 4;
    op.max_vec = vec_of_align(req->align);
    if (op.max_vec < dsz) return GBX_ERR_UNSUPPORTED;
    op.min_vec = req->forced_vec ? std::max(dsz, std::min(req->forced_vec, op.max_vec)) : std::max(dsz, op.max_vec / 2);
    if (req->forced_vec) op.max_vec = op.min_vec;
    op.block = 256;
    op.persistent = 1;
    const int64_t s = req->elem_size;
    // per row: its 16-byte record, its output element (read too when accumulating); per term:
    // the gradient element, plus the 8-byte term entry for rows with more than one term
    op.algo_bytes = nterms * s + nrows * s * (accumulate ? 2 : 1) + nrows * 16 + (nterms - nrows) * 8;
    op.idx_len = nterms;
    FoldDesc &d = op.fd;
    d.out = out; d.bufA = bufA; d.bufB = bufB; d.row_ptr = row_ptr; d.row_out = row_out; d.terms = terms;
    d.nrows = nrows; d.elem_size = s; d.dtype = req->dtype; d.accumulate = accumulate;
    d.out_role = out_role; d.a_role = a_role; d.b_role = b_role;
    d.status = req->status_dev; d.wait_limit = req->wait_limit;
    const int64_t max_tiles = ceil_div(nrows * (s / op.min_vec), GBX_TILE);
    GBX_TRY(req->mem.get(&op.d_tile_e0, max_tiles + 1));
    d.tile_e0 = op.d_tile_e0;
    GBX_TRY(req->mem.get(&op.d_rec, nrows));
    GBX_TRY(gbx_build_fold_records(row_ptr, row_out, terms, nrows, op.d_rec, req->stream));
    d.rec = op.d_rec;
    // the stream form copies records (16-byte entries) and term lists rounded out to 16 bytes
    // (every term array the library builds is 16-byte aligned with 2 entries of padding)
    {
        static int prepared = 0;
        op.sfold_ok = req->allow_stream && !(((uintptr_t)terms | (uintptr_t)op.d_rec) & 15);
        if (op.sfold_ok && !prepared) {
            if (gbx_sfold_prepare() == GBX_SUCCESS) prepared = 1;
            else op.sfold_ok = 0;
        }
    }
    GBX_TRY(req->mem.alloc(&op.d_desc, sizeof(FoldDesc)));
    GBX_TRY(req->mem.get(&op.d_self, 1));
    GBX_TRY(req->mem.get(&op.d_self_prefix, 2));
    req->ops.push_back(op);
    return GBX_SUCCESS;
}

static int64_t op_tiles(const HostOp &op) { return op.kind == 0 ? op.cd.ntiles : op.fd.ntiles; }

static int upload_desc(gbx_request_s *req, HostOp &op) {
    if (op.kind == 0)
        GBX_CUDA_TRY(cudaMemcpyAsync(op.d_desc, &op.cd, sizeof(CopyDesc), cudaMemcpyHostToDevice, req->stream));
    else
        GBX_CUDA_TRY(cudaMemcpyAsync(op.d_desc, &op.fd, sizeof(FoldDesc), cudaMemcpyHostToDevice, req->stream));
    return GBX_SUCCESS;
}

// Sets the op's vector width: chunk geometry, tiles, tile->segment table, descriptor.
static int set_vec(gbx_request_s *req, HostOp &op, int vec) {
    const int64_t s = req->elem_size;
    // the tile tables were allocated for min_vec; a narrower vector would need more tiles
    if (vec < op.min_vec || vec > op.max_vec) return GBX_ERR_INTERNAL;
    const int cpe = (int)(s / vec);
    int shift = -1;
    if ((cpe & (cpe - 1)) == 0) { shift = 0; while ((1 << shift) < cpe) shift++; }
    const uint32_t magic = shift >= 0 ? 0u : (uint32_t)(((1ull << 32) + (uint64_t)cpe - 1) / (uint64_t)cpe);
    if (op.kind == 0) {
        CopyDesc &d = op.cd;
        d.vec = vec; d.cpe = cpe; d.cpe_shift = shift; d.cpe_magic = magic;
        d.nchunks = d.nelem * cpe;
        d.ntiles = ceil_div(d.nchunks, GBX_TILE);
        if (d.flat == 8)   // bulk form: one "tile" per piece, no tile table
            d.ntiles = d.nbulk;
        else if (d.flat == 9)   // scatter form: one "tile" per source window
            d.ntiles = d.nscat;
        else if (op.flat_only)
            GBX_TRY(gbx_build_tile_meta(nullptr, 0, cpe, d.ntiles, nullptr, op.d_tile_e0, req->stream));
        else
            GBX_TRY(gbx_build_tile_meta(d.segs, d.nseg, cpe, d.ntiles, op.d_tile_seg, op.d_tile_e0, req->stream));
    } else {
        FoldDesc &d = op.fd;
        d.vec = vec; d.cpe = cpe; d.cpe_shift = shift; d.cpe_magic = magic;
        d.nchunks = d.nrows * cpe;
        d.ntiles = ceil_div(d.nchunks, GBX_TILE);
        GBX_TRY(gbx_build_tile_meta(nullptr, 0, cpe, d.ntiles, nullptr, op.d_tile_e0, req->stream));
    }
    GBX_TRY(upload_desc(req, op));
    void *self = op.d_desc;
    int64_t pre[2] = {0, op_tiles(op)};
    GBX_CUDA_TRY(cudaMemcpyAsync(op.d_self, &self, sizeof(void *), cudaMemcpyHostToDevice, req->stream));
    GBX_CUDA_TRY(cudaMemcpyAsync(op.d_self_prefix, pre, sizeof(pre), cudaMemcpyHostToDevice, req->stream));
    GBX_CUDA_TRY(cudaStreamSynchronize(req->stream));
    return GBX_SUCCESS;
}

static int op_vec(const HostOp &op) { return op.kind == 0 ? op.cd.vec : op.fd.vec; }

// Grid of a launch: one block per tile, or persistent (SMs x resident blocks); at most
// max_ctas blocks when that is set (every move kernel walks its tiles grid-stride, so any
// grid covers them), which leaves room for other requests' kernels on other streams.
static int grid_for(int kind, int dtype, int vec, int flat, int block, int persistent, int64_t tiles,
                    int max_ctas) {
    if ((kind == 0 && flat >= 10) || (kind == 1 && flat == 1)) persistent = 1;   // stream kernels: resident rings
    int64_t g = persistent ? (int64_t)gbx_num_sms() * gbx_occupancy(kind, dtype, vec, block, flat)
                           : std::min<int64_t>(tiles, 1ll << 30);
    if (max_ctas > 0) g = std::min<int64_t>(g, max_ctas);
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, tiles));
}

// one: every op of the launch has one chunk per element (the stream forms then run their
// specialised kernel, launch codes 12 / 13)
static cudaError_t launch_list(int kind, int dtype, int vec, int flat, void **d_ops, int64_t *d_prefix, int nops,
                               int64_t tiles, int block, int grid, cudaStream_t st, int one = 0) {
    if (kind == 0)
        return gbx_launch_copy((const CopyDesc *const *)d_ops, d_prefix, nops, tiles, vec,
                               (flat == 10 || flat == 11) && one ? flat + 2 : flat, block, grid, st);
    return gbx_launch_fold((const FoldDesc *const *)d_ops, d_prefix, nops, tiles, dtype, vec, block, grid, st, flat);
}

// a copy's form, or a fold's (0 the fold kernel, 1 its stream form)
static int op_flat(const HostOp &op) { return op.kind == 0 ? op.cd.flat : op.fold_form; }

static cudaError_t launch_op_alone(gbx_request_s *req, HostOp &op, int block, int persistent) {
    int64_t tiles = op_tiles(op);
    const int vec = op_vec(op), flat = op_flat(op);
    return launch_list(op.kind, req->dtype, vec, flat, op.d_self, op.d_self_prefix, 1, tiles, block,
                       grid_for(op.kind, req->dtype, vec, flat, block, persistent, tiles, req->max_ctas), req->stream,
                       op.kind == 0 && op.cd.cpe == 1);
}

// ------------------------------------------------------------------ autotuner
// Times every candidate shape of an op (vector width, block size, grid mode) with
// CUDA events on the request's stream and keeps the fastest.  Results never depend on
// the shape: every candidate moves the same bytes to the same places.  Chosen shapes are
// cached by a signature of the op, so identical patterns are tuned once per process.
struct TuneKey {
    int kind, max_vec, min_vec, dtype, flat_ok;
    int64_t units, nseg, elem_size, nterms;
    bool operator<(const TuneKey &o) const {
        return memcmp(this, &o, sizeof(TuneKey)) < 0;
    }
};
struct TuneVal { int vec, block, persistent, flat; float ms; };
static std::map<TuneKey, TuneVal> g_tune_cache;
static std::mutex g_tune_mu;

static int time_op(gbx_request_s *req, HostOp &op, int block, int persistent, int reps, float *ms) {
    cudaEvent_t a, b;
    GBX_CUDA_TRY(cudaEventCreate(&a));
    GBX_CUDA_TRY(cudaEventCreate(&b));
    cudaError_t e = launch_op_alone(req, op, block, persistent);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; r++) {
        cudaEventRecord(a, req->stream);
        e = launch_op_alone(req, op, block, persistent);
        cudaEventRecord(b, req->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
        best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) {
        gbx_note_cuda_error(e, "tuning launch", __FILE__, __LINE__);
        return GBX_ERR_CUDA;
    }
    *ms = best;
    return GBX_SUCCESS;
}

// algorithmic bytes of a copy in the form it runs in
static void set_form_bytes(HostOp &op) {
    if (op.kind != 0) return;
    op.algo_bytes = op.cd.flat == 8 ? op.algo_bytes_bulk
                  : op.cd.flat == 9 ? op.algo_bytes_scat
                  : op.cd.flat ? op.algo_bytes_flat : op.algo_bytes_seg;
}

static int tune_op(gbx_request_s *req, HostOp &op) {
    TuneKey key;
    memset(&key, 0, sizeof(key));
    key.kind = op.kind; key.max_vec = op.max_vec; key.min_vec = op.min_vec; key.dtype = req->dtype;
    key.units = op.units; key.elem_size = req->elem_size;
    key.nseg = op.kind == 0 ? op.cd.nseg : 0;
    key.nterms = op.kind == 1 ? op.fd.nchunks : 0;
    key.flat_ok = op.kind == 1 ? op.sfold_ok + 2 * (req->forced_form + 1)
                : op.kind == 0 ? op.flat_ok + 2 * op.flat_only + 4 * ((op.cd.flat & 3) == 3) + 8 * op.bulk_ok +
                                     16 * op.scat_ok + 32 * (req->allow_bulk == 2) + 64 * op.stream_ok +
                                     128 * (req->allow_stream == 2) + 256 * (req->forced_form + 1)   // forced forms tune apart
                : 0;
    int blocks[4] = {128, 256, 512, 1024};
    if (!req->autotune || req->forced_block) {
        op.block = req->forced_block ? req->forced_block : 256;
        op.persistent = 1;
        if (op.kind == 1) op.fold_form = op.sfold_ok && req->allow_stream == 2;
        if (op.kind == 0 && !op.flat_only) op.cd.flat = op.flat_ok && req->forced_flat != 0;
        if (op.kind == 0 && op.stream_ok && req->allow_stream == 2) op.cd.flat = (op.cd.flat & 3) == 3 ? 11 : 10;
        if (op.kind == 0 && op.bulk_ok && req->allow_bulk == 2) op.cd.flat = 8;
        if (op.kind == 0 && op.scat_ok && req->allow_bulk == 2) op.cd.flat = 9;
        set_form_bytes(op);
        return set_vec(req, op, op.max_vec);
    }
    if (op.kind == 1 && op.fd.accumulate) {
        // an accumulating fold adds into the caller's buffer, so it is never trial-launched:
        // it takes the shape tuned for the same rows without accumulation, or the default
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        op.block = it != g_tune_cache.end() ? it->second.block : 256;
        op.persistent = it != g_tune_cache.end() ? it->second.persistent : 1;
        op.fold_form = it != g_tune_cache.end() ? it->second.flat : 0;
        return set_vec(req, op, it != g_tune_cache.end() ? it->second.vec : op.max_vec);
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            op.block = it->second.block;
            op.persistent = it->second.persistent;
            op.tuned_ms = it->second.ms;
            if (op.kind == 0) op.cd.flat = it->second.flat;
            else op.fold_form = it->second.flat;
            set_form_bytes(op);
            return set_vec(req, op, it->second.vec);
        }
    }
    TuneVal best = {op.max_vec, 256, 1, 0, 1e30f};
    // candidate forms: segments, flat (gather or two-index), and the pipelined flat form
    std::vector<int> forms;
    if (op.kind == 1) {
        forms.push_back(0);
        if (op.sfold_ok) forms.push_back(1);   // the fold's stream form
        if (op.sfold_ok && (req->allow_stream == 2 || req->forced_form == 1)) forms.assign(1, 1);
    }
    else if (op.flat_only) { forms.push_back(op.cd.flat & 3); forms.push_back((op.cd.flat & 3) + 4); }
    else if (op.flat_ok && req->forced_flat < 0) { forms.push_back(0); forms.push_back(1); forms.push_back(5); }
    else if (op.flat_ok && req->forced_flat > 0) { forms.push_back(1); forms.push_back(5); }
    else forms.push_back(0);
    if (op.kind == 0 && op.stream_ok && (op.flat_only || (op.flat_ok && req->forced_flat != 0)))
        forms.push_back((op.cd.flat & 3) == 3 ? 11 : 10);
    // (bulk_ok implies 16-byte aligned pieces; between the library's own aggregates the element
    // size need not be a multiple of 16)
    if (op.kind == 0 && op.bulk_ok && req->forced_flat != 1) forms.push_back(8);
    if (op.kind == 0 && op.scat_ok && op.max_vec == 16) forms.push_back(9);
    if (op.kind == 0 && op.stream_ok && req->allow_stream == 2) forms.assign(1, (op.cd.flat & 3) == 3 ? 11 : 10);
    if (op.kind == 0 && op.bulk_ok && req->allow_bulk == 2) forms.assign(1, 8);   // forced where it applies
    if (op.kind == 0 && op.scat_ok && req->allow_bulk == 2) forms.assign(1, 9);
    if (op.kind == 0 && req->forced_form >= 0 &&   // one form, where the op offers it
        std::find(forms.begin(), forms.end(), req->forced_form) != forms.end())
        forms.assign(1, req->forced_form);
    for (int form : forms) {
        if (op.kind == 0) op.cd.flat = form;
        else op.fold_form = form;
        const bool pipe = op.kind == 0 && form >= 4 && form < 8, bulk = op.kind == 0 && (form == 8 || form == 9);
        const bool strm = op.kind == 0 ? form >= 10 : form == 1;
        // (the op's tile tables are sized for min_vec: no width below it)
        // (the bulk and scatter kernels do not use the vector width: one pass, at max_vec)
        for (int vec = op.max_vec; vec >= (bulk ? op.max_vec : strm ? std::max(4, op.min_vec) : op.min_vec);
             vec >>= 1) {
            GBX_TRY(set_vec(req, op, vec));
            // stream forms: persistent grid only; block 256 and 512 select the two wide shapes,
            // block 128 the narrow one, offered only with one chunk per element (cpe == 1)
            const int b0 = pipe ? 2 : form == 8 ? 3 : strm ? (op.kind == 0 && op.cd.cpe == 1 && vec <= 8 ? 0 : 1) : 0;
            for (int bi = b0; bi < (strm ? 3 : 4); bi++)
                for (int pers = 1; pers >= (pipe || strm ? 1 : 0); pers--) {
                    float ms = 0;
                    GBX_TRY(time_op(req, op, blocks[bi], pers, 3, &ms));
                    // a narrower vector must win clearly: it adds a kernel class to any batch
                    // the op joins, and small ops (under two waves of tiles) time within noise
                    const float margin = op_tiles(op) < 2 * 4 * gbx_num_sms() ? 0.85f : 0.97f;
                    // the bulk form wins near-ties: it reads no per-element index and leaves the
                    // SMs' load / store issue to the copy engine (repeated trials with a warm L2
                    // time the index-driven forms within a few per cent of it)
                    if (op.kind == 0 && form == 8) ms *= 0.97f;
                    if (ms < best.ms * (vec < best.vec ? margin : 1.0f)) best = {vec, blocks[bi], pers, form, ms};
                }
            if (vec == 1) break;
        }
    }
    op.block = best.block;
    op.persistent = best.persistent;
    op.tuned_ms = best.ms;
    if (op.kind == 0) op.cd.flat = best.flat;
    else op.fold_form = best.flat;
    set_form_bytes(op);
    GBX_TRY(set_vec(req, op, best.vec));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return GBX_SUCCESS;
}

// ------------------------------------------------------- levels and the graph
// One launch per (level, kind, class): a class is (form, vector width) for copies and
// (payload type, vector width) for folds, so every launch runs a specialised kernel.  For a
// batch the ops of all its requests are pooled, so each launch covers every pattern of its
// class (the generic width-dispatching kernels stay available but are not needed).
// Times a pooled launch in every block size and grid mode with CUDA events and keeps the
// fastest (the moved bytes do not depend on the shape).
static int tune_launch(LevelLaunch &L, cudaStream_t st) {
    cudaEvent_t a, b;
    GBX_CUDA_TRY(cudaEventCreate(&a));
    GBX_CUDA_TRY(cudaEventCreate(&b));
    const int blocks[4] = {128, 256, 512, 1024};
    float best = 1e30f;
    int bb = L.block, bg = L.grid, bf = L.flat;
    cudaError_t e = cudaSuccess;
    // a stream-form launch is also timed in the plain flat form (same tiles, same bytes)
    const int nforms = (L.flat == 10 || L.flat == 11) ? 2 : 1;
    for (int fi = 0; fi < nforms && e == cudaSuccess; fi++) {
        const int fl = fi == 0 ? L.flat : (L.flat == 10 ? 1 : 3);
        const bool strm = fl >= 10;
        for (int bi = strm ? (L.one && L.vec <= 8 ? 0 : 1) : 0; bi < (strm ? 3 : 4) && e == cudaSuccess; bi++)
            for (int pers = 1; pers >= (strm ? 1 : 0) && e == cudaSuccess; pers--) {
                const int blk = gbx_effective_block(L.vec, blocks[bi]);
                const int grid = grid_for(L.kind, L.dtype, L.vec, fl, blk, pers, L.total_tiles, L.max_ctas);
                e = launch_list(L.kind, L.dtype, L.vec, fl, L.d_ops, L.d_prefix, L.nops, L.total_tiles, blk, grid, st,
                                L.one);
                float t = 1e30f;
                for (int r = 0; r < 3 && e == cudaSuccess; r++) {
                    cudaEventRecord(a, st);
                    e = launch_list(L.kind, L.dtype, L.vec, fl, L.d_ops, L.d_prefix, L.nops, L.total_tiles, blk,
                                    grid, st, L.one);
                    cudaEventRecord(b, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    float x = 0;
                    if (e == cudaSuccess) cudaEventElapsedTime(&x, a, b);
                    t = std::min(t, x);
                }
                if (t < best) { best = t; bb = blk; bg = grid; bf = fl; }
            }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) {
        gbx_note_cuda_error(e, "tuning a pooled launch", __FILE__, __LINE__);
        return GBX_ERR_CUDA;
    }
    L.block = bb;
    L.grid = bg;
    L.flat = bf;
    return GBX_SUCCESS;
}

// NVTX name of a launch: what = 0 standard forward, 1 locality forward (levels = its three
// steps), 2 backward, 3 batch.
static const char *phase_name(int what, int level, int kind) {
    static const char *const fwd_loc[3] = {"gbx.locality.step1_gather", "gbx.locality.step2_node_pairs",
                                           "gbx.locality.step3_redistribute"};
    static const char *const bwd[2][3] = {{"gbx.backward.level0.copy", "gbx.backward.level1.copy",
                                           "gbx.backward.level2.copy"},
                                          {"gbx.backward.level0.fold", "gbx.backward.level1.fold",
                                           "gbx.backward.level2.fold"}};
    static const char *const bat[2][3] = {{"gbx.batch.level0.copy", "gbx.batch.level1.copy", "gbx.batch.level2.copy"},
                                          {"gbx.batch.level0.fold", "gbx.batch.level1.fold", "gbx.batch.level2.fold"}};
    const int lv = level < 0 ? 0 : level > 2 ? 2 : level, k = kind ? 1 : 0;
    switch (what) {
        case 0: return "gbx.standard.move";
        case 1: return fwd_loc[lv];
        case 2: return bwd[k][lv];
        default: return bat[k][lv];
    }
}

static int build_levels(DevPool &mem, const std::vector<HostOp *> &ops, const std::vector<int> &dtypes,
                        std::vector<LevelLaunch> &out, int batch, cudaStream_t st, int tune = 0, int max_ctas = 0,
                        int what = 3) {
    int nlev = 0;
    for (HostOp *op : ops) nlev = std::max(nlev, op->level + 1);
    for (int lv = 0; lv < nlev; lv++)
        for (int kind = 0; kind < 2; kind++) {
            std::vector<std::vector<size_t>> groups;
            std::vector<std::pair<int, int>> keys;   // (dtype or form, vec) of each group
            for (size_t i = 0; i < ops.size(); i++) {
                HostOp *op = ops[i];
                if (op->level != lv || op->kind != kind || op_tiles(*op) <= 0) continue;
                // every launch is specialised: ops are grouped by (form, vector width) for copies
                // and (payload type, vector width) for folds; a batch fuses all patterns of a
                // class, with every copy that has the flat form in one flat launch whatever form
                // it was tuned to alone (fewer, larger launches)
                // bulk / scatter ops pool only with their own kind (their tiles are pieces); every
                // other flat-capable op joins the stream-form launch when all its index arrays allow
                // it, else the plain flat launch
                const int f0 = op_flat(*op);
                const bool strm = op->stream_ok && op_vec(*op) >= 4;
                const int form = !batch || f0 == 8 || f0 == 9 ? f0
                               : op->flat_ok ? ((f0 & 3) == 3 ? (strm ? 11 : 3) : (strm ? 10 : 1)) : 0;
                // stream-form copies with one chunk per element get a launch of their own, which
                // runs the specialised kernel (one op with more chunks would hold back the rest)
                const int one = kind == 0 && form >= 10 && op->cd.cpe == 1 ? 16 : 0;
                std::pair<int, int> k = kind ? std::make_pair(dtypes[i] + 8 * op->fold_form, op_vec(*op))
                                             : std::make_pair(form + one, op_vec(*op));
                size_t g = 0;
                while (g < keys.size() && keys[g] != k) g++;
                if (g == keys.size()) { keys.push_back(k); groups.emplace_back(); }
                groups[g].push_back(i);
            }
            for (size_t g = 0; g < groups.size(); g++) {
                LevelLaunch L;
                L.kind = kind;
                L.nops = (int)groups[g].size();
                // common payload type, vector width and form, or 0 / 2 (= mixed)
                int dt = dtypes[groups[g][0]], vec = op_vec(*ops[groups[g][0]]);
                // (a pooled class of one op keeps the form it was tuned to, pipelined included)
                int fl = kind ? ops[groups[g][0]]->fold_form
                              : (groups[g].size() == 1 ? op_flat(*ops[groups[g][0]]) : keys[g].first & 15);
                for (size_t i : groups[g]) {
                    if (dtypes[i] != dt) dt = -1;
                    if (op_vec(*ops[i]) != vec) vec = 0;
                    if (!batch && op_flat(*ops[i]) != fl) fl = 2;
                }
                if (dt < 0 && kind == 1) vec = 0;
                L.dtype = dt < 0 ? GBX_F32 : dt;
                L.vec = vec;
                L.flat = vec == 0 ? 2 : fl;
                L.one = 1;
                for (size_t i : groups[g])
                    if (kind != 0 || ops[i]->cd.cpe != 1) L.one = 0;
                std::vector<void *> ptrs;
                std::vector<int64_t> pre(1, 0);
                const HostOp *big = ops[groups[g][0]];
                for (size_t i : groups[g]) {
                    ptrs.push_back(ops[i]->d_desc);
                    pre.push_back(pre.back() + op_tiles(*ops[i]));
                    if (op_tiles(*ops[i]) > op_tiles(*big)) big = ops[i];
                }
                L.total_tiles = pre.back();
                L.phase = phase_name(batch ? 3 : what, lv, kind);
                // the launch takes the tuned shape of its largest op
                L.block = gbx_effective_block(L.vec, big->block);
                L.max_ctas = max_ctas;
                L.grid = grid_for(kind, L.dtype, L.vec, L.flat, L.block, big->persistent, L.total_tiles, max_ctas);
                GBX_TRY(mem.get(&L.d_ops, L.nops));
                GBX_TRY(mem.get(&L.d_prefix, L.nops + 1));
                GBX_CUDA_TRY(cudaMemcpyAsync(L.d_ops, ptrs.data(), sizeof(void *) * ptrs.size(),
                                             cudaMemcpyHostToDevice, st));
                GBX_CUDA_TRY(cudaMemcpyAsync(L.d_prefix, pre.data(), sizeof(int64_t) * pre.size(),
                                             cudaMemcpyHostToDevice, st));
                // a pooled copy launch of a batch is tuned as a whole (copies only: a trial
                // writes the bytes the real launch writes next; folds keep their op's shape)
                if (batch && kind == 0 && L.nops > 1 && tune) GBX_TRY(tune_launch(L, st));
                out.push_back(L);
            }
        }
    GBX_CUDA_TRY(cudaStreamSynchronize(st));
    return GBX_SUCCESS;
}

static cudaError_t enqueue_levels(const std::vector<LevelLaunch> &levels, cudaStream_t st) {
    for (const LevelLaunch &L : levels) {
        GbxRange r(L.phase);
        cudaError_t e = launch_list(L.kind, L.dtype, L.vec, L.flat, L.d_ops, L.d_prefix, L.nops, L.total_tiles,
                                    L.block, L.grid, st, L.one);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int capture(const std::vector<LevelLaunch> &levels, cudaGraphExec_t *exec) {
    cudaStream_t cs;
    GBX_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_levels(levels, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        gbx_note_cuda_error(e, "graph capture", __FILE__, __LINE__);
        return GBX_ERR_CUDA;
    }
    return GBX_SUCCESS;
}

static void fill_info(gbx_request_s *req) {
    gbx_request_info_t &I = req->info;
    I.kind = req->kind;
    I.algorithm = req->algorithm;
    int nlev = 0;
    int64_t algo = 0;
    const HostOp *big = nullptr;
    I.copy_forms = 0;
    for (const HostOp &op : req->ops) {
        nlev = std::max(nlev, op.level + 1);
        algo += op.algo_bytes;
        if (op.kind == 0) I.copy_forms |= (int64_t)1 << op.cd.flat;
        else if (op.fold_form) I.copy_forms |= (int64_t)1 << 12;   // a fold in its stream form
        if (!big || op.algo_bytes > big->algo_bytes) big = &op;
    }
    I.levels = nlev;
    I.launches = (int)req->launches.size();
    I.use_graph = req->use_graph;
    I.algo_bytes = algo;
    if (big) {
        I.vec_bytes = big->kind == 0 ? big->cd.vec : big->fd.vec;
        I.block = big->block;
        I.unroll = GBX_TILE / big->block;
    }
    I.device_bytes = req->mem.bytes;
}

static int finalize(gbx_request_s *req) {
    {
        GbxRange r("gbx.setup.validate");
        GBX_TRY(gbx_validate_program(req, req->agg ? 2 * req->Ur * req->elem_size : 0));
    }
    {
        GbxRange r("gbx.setup.tune");
        for (HostOp &op : req->ops) GBX_TRY(tune_op(req, op));
    }
    GbxRange r("gbx.setup.capture");
    std::vector<HostOp *> ptrs;
    std::vector<int> dts;
    for (HostOp &op : req->ops) { ptrs.push_back(&op); dts.push_back(req->dtype); }
    const int what = req->kind == 1 ? 2 : req->algorithm == GBX_ALG_LOCALITY ? 1 : 0;
    GBX_TRY(build_levels(req->mem, ptrs, dts, req->launches, 0, req->stream, 0, req->max_ctas, what));
    if (req->use_graph && !req->launches.empty()) GBX_TRY(capture(req->launches, &req->exec));
    fill_info(req);
    return GBX_SUCCESS;
}

static void destroy_batch(Batch *b) {
    for (gbx_request_s *m : b->members) {
        auto &v = m->batches;
        v.erase(std::remove(v.begin(), v.end(), b), v.end());
        if (m->pending == &b->done) {
            cudaEventSynchronize(b->done);
            m->pending = nullptr;
            m->active = 0;
        }
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

static void destroy_request(gbx_request_s *req) {
    if (!req) return;
    if (req->kind == 2) {
        for (size_t k = 0; k < req->part_ev.size(); k++) {
            if (req->part_ready[k]) cudaEventSynchronize(req->part_ev[k]);
            cudaEventDestroy(req->part_ev[k]);
        }
        for (gbx_request_s *c : req->parts) destroy_request(c);
        req->parts.clear();
        req->active = 0;
    }
    if (req->active) {
        cudaEvent_t ev = req->pending ? *req->pending : req->done;
        cudaEventSynchronize(ev);
    }
    while (!req->batches.empty()) destroy_batch(req->batches.back());
    if (req->host_down_pending) cudaEventSynchronize(req->host_down_ev);
    if (req->host_up) cudaStreamSynchronize(req->host_up);
    for (cudaEvent_t e : {req->host_up_ev, req->host_down_ev, req->host_mark})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : {req->host_up, req->host_down})
        if (s) cudaStreamDestroy(s);
    if (req->exec) cudaGraphExecDestroy(req->exec);
    if (req->done) cudaEventDestroy(req->done);
    if (req->status_host) cudaFreeHost(req->status_host);
    gbx_graph_s *g = req->owned_graph;
    delete req;
    if (g) gbx_graph_free(&g);
}

// Events that other streams wait on (cudaStreamWaitEvent: gbx_wait_stream, gbx_parrived_stream,
// the host-buffer copy streams, batches) are created with timing enabled: on GB300 a stream
// waiting on a disable-timing event held back the work queued behind the wait (an early-bird
// exchange of 8 partitions took 2.99 ms against 2.47 ms with timing-enabled events).
static cudaError_t gbx_event_create(cudaEvent_t *ev) { return cudaEventCreateWithFlags(ev, cudaEventDefault); }

static gbx_request_s *new_request(const Opts &o, void *stream) {
    gbx_request_s *req = new gbx_request_s();
    cudaGetDevice(&req->device);
    req->stream = (cudaStream_t)stream;
    req->use_graph = o.graph;
    req->autotune = o.autotune;
    req->forced_vec = o.vec;
    req->forced_block = o.block;
    req->timeout_ms = o.timeout_ms;
    req->min_run = o.min_run;
    req->piece = o.piece;
    req->forced_flat = o.flat;
    req->allow_flat = o.flat != 0;
    req->no_combine = o.flat == 0;
    req->no_single_split = !o.split;
    req->split_order = o.split_order;
    req->check_dup = o.check_dup;
    req->allow_bulk = o.bulk;
    req->max_ctas = o.max_ctas;
    req->wait_limit = o.wait_limit;
    req->allow_stream = o.stream;
    req->forced_form = o.form;
    if (gbx_event_create(&req->done) != cudaSuccess) {
        cudaGetLastError();
        req->done = nullptr;
    }
    // the status word (a failed allocation leaves the request unusable: done = null)
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped) != cudaSuccess || cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaGetLastError();
        if (h) cudaFreeHost(h);
        if (req->done) cudaEventDestroy(req->done);
        req->done = nullptr;
    } else {
        memset(h, 0, 64);
        req->status_host = (int *)h;
        req->status_dev = (int *)d;
    }
    return req;
}

static float program_ms(gbx_request_s *req) {
    // time of one eager pass over the levels (used by algorithm=auto)
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return 1e30f;
    enqueue_levels(req->launches, req->stream);
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
        cudaEventRecord(a, req->stream);
        enqueue_levels(req->launches, req->stream);
        cudaEventRecord(b, req->stream);
        cudaEventSynchronize(b);
        float t = 0;
        cudaEventElapsedTime(&t, a, b);
        best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

extern "C" int gbx_neighbor_alltoallv_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                           const int *sendcounts, const int *sdispls, const int64_t *send_slot_ptr,
                                           const int *send_idx, void *recvbuf, int64_t recvbuf_bytes,
                                           const int64_t *recv_base, const int *recvcounts, const int *rdispls,
                                           const int64_t *recv_slot_ptr, int64_t elem_size, int dtype,
                                           const int64_t *global_sidx, const int64_t *global_ridx, gbx_graph_t graph,
                                           const char *info, void *stream, gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!graph || elem_size <= 0 || sendbuf_bytes < 0 || recvbuf_bytes < 0) return GBX_ERR_ARG;
    if (dtype != GBX_BYTES && dtype != GBX_F32 && dtype != GBX_F64) return GBX_ERR_ARG;
    if ((sendbuf_bytes > 0 && !sendbuf) || (recvbuf_bytes > 0 && !recvbuf)) return GBX_ERR_ARG;
    if (!send_base || !recv_base) return GBX_ERR_ARG;
    if (graph->E > 0 && (!sendcounts || !sdispls || !recvcounts || !rdispls)) return GBX_ERR_ARG;
    GBX_TRY(gbx_check_data_buf(sendbuf, sendbuf_bytes));
    GBX_TRY(gbx_check_data_buf(recvbuf, recvbuf_bytes));
    if ((send_idx || global_sidx) && !send_slot_ptr) return GBX_ERR_ARG;
    if (global_ridx && (!recv_slot_ptr || !global_sidx)) return GBX_ERR_ARG;
    Opts o = parse_info(info);
    if (!o.ok) return GBX_ERR_ARG;

    auto build = [&](int locality, gbx_request_s **out) -> int {
        GbxRange range(locality ? "gbx.setup.forward_locality" : "gbx.setup.forward_standard");
        gbx_request_s *req = new_request(o, stream);
        if (!req->done) { destroy_request(req); return GBX_ERR_CUDA; }
        req->kind = 0;
        req->graph = graph;
        req->src = (const char *)sendbuf;
        req->dst = (char *)recvbuf;
        req->src_bytes = sendbuf_bytes;
        req->dst_bytes = recvbuf_bytes;
        req->elem_size = elem_size;
        req->dtype = dtype;
        int rc = gbx_setup_forward(req, send_base, sendcounts, sdispls, send_slot_ptr, send_idx, recv_base,
                                   recvcounts, rdispls, recv_slot_ptr, global_sidx, global_ridx, locality);
        if (rc == GBX_SUCCESS) rc = finalize(req);
        if (rc != GBX_SUCCESS) { destroy_request(req); return rc; }
        *out = req;
        return GBX_SUCCESS;
    };

    gbx_request_s *req = nullptr;
    if (o.algorithm_auto) {
        gbx_request_s *a = nullptr, *b = nullptr;
        GBX_TRY(build(0, &a));
        int rc = build(1, &b);
        if (rc != GBX_SUCCESS) { destroy_request(a); return rc; }
        float ta = program_ms(a), tb = program_ms(b);
        if (tb < ta) { destroy_request(a); req = b; }
        else { destroy_request(b); req = a; }
    } else {
        GBX_TRY(build(o.algorithm == GBX_ALG_LOCALITY, &req));
    }
    *request = req;
    return GBX_SUCCESS;
}

extern "C" int gbx_neighbor_alltoallw_init(const void *sendbuf, int64_t sendbuf_bytes, const int64_t *send_base,
                                           const int *sendcounts, const int64_t *sdispls, const int *sendtypes,
                                           void *recvbuf, int64_t recvbuf_bytes, const int64_t *recv_base,
                                           const int *recvcounts, const int64_t *rdispls, const int *recvtypes,
                                           const gbx_datatype_t *types, int ntypes, int dtype, gbx_graph_t graph,
                                           const char *info, void *stream, gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!graph || sendbuf_bytes < 0 || recvbuf_bytes < 0 || ntypes < 0 || (ntypes > 0 && !types)) return GBX_ERR_ARG;
    if (dtype != GBX_BYTES && dtype != GBX_F32 && dtype != GBX_F64) return GBX_ERR_ARG;
    if ((sendbuf_bytes > 0 && !sendbuf) || (recvbuf_bytes > 0 && !recvbuf)) return GBX_ERR_ARG;
    if (!send_base || !recv_base) return GBX_ERR_ARG;
    if (graph->E > 0 && (!sendcounts || !sdispls || !sendtypes || !recvcounts || !rdispls || !recvtypes))
        return GBX_ERR_ARG;
    GBX_TRY(gbx_check_data_buf(sendbuf, sendbuf_bytes));
    GBX_TRY(gbx_check_data_buf(recvbuf, recvbuf_bytes));
    Opts o = parse_info(info);
    if (!o.ok) return GBX_ERR_ARG;
    if (o.algorithm != GBX_ALG_STANDARD || o.algorithm_auto) return GBX_ERR_UNSUPPORTED;
    GbxRange range("gbx.setup.alltoallw");
    gbx_request_s *req = new_request(o, stream);
    if (!req->done) { destroy_request(req); return GBX_ERR_CUDA; }
    req->kind = 0;
    req->graph = graph;
    req->src = (const char *)sendbuf;
    req->dst = (char *)recvbuf;
    req->src_bytes = sendbuf_bytes;
    req->dst_bytes = recvbuf_bytes;
    req->dtype = dtype;
    int rc = gbx_setup_alltoallw(req, send_base, sendcounts, sdispls, sendtypes, recv_base, recvcounts, rdispls,
                                 recvtypes, types, ntypes);
    if (rc == GBX_SUCCESS) rc = finalize(req);
    if (rc != GBX_SUCCESS) { destroy_request(req); return rc; }
    *request = req;
    return GBX_SUCCESS;
}

// ------------------------------------------------------------ partitioned
static int check_part_ptr(int n, const int64_t *ptr, int64_t bytes) {
    if (n < 1 || n > 1024 || !ptr || ptr[0] != 0 || ptr[n] != bytes) return GBX_ERR_ARG;
    for (int k = 0; k < n; k++)
        if (ptr[k + 1] < ptr[k]) return GBX_ERR_ARG;
    return GBX_SUCCESS;
}

extern "C" int gbx_partitioned_init(gbx_request_t forward, int npart, const int64_t *part_ptr, int nrpart,
                                    const int64_t *rpart_ptr, const char *info, void *stream,
                                    gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!forward || forward->kind != 0) return GBX_ERR_ARG;
    if (forward->algorithm != GBX_ALG_STANDARD) return GBX_ERR_UNSUPPORTED;
    GBX_TRY(check_part_ptr(npart, part_ptr, forward->src_bytes));
    GBX_TRY(check_part_ptr(nrpart, rpart_ptr, forward->dst_bytes));
    Opts o = parse_info(info);
    if (!o.ok) return GBX_ERR_ARG;
    GbxRange range("gbx.setup.partitioned");
    gbx_request_s *req = new_request(o, stream);
    if (!req->done) { destroy_request(req); return GBX_ERR_CUDA; }
    req->kind = 2;
    req->forward = forward;
    req->graph = forward->graph;
    req->src = forward->src;
    req->dst = forward->dst;
    req->src_bytes = forward->src_bytes;
    req->dst_bytes = forward->dst_bytes;
    req->elem_size = forward->elem_size;
    req->dtype = forward->dtype;
    req->align = forward->align;
    req->algorithm = GBX_ALG_STANDARD;
    req->npart = npart;
    req->nrpart = nrpart;
    req->part_ready.assign(npart, 0);
    PartPlan plan;
    int rc = gbx_setup_partitions(req, forward, npart, part_ptr, nrpart, rpart_ptr, &plan);
    const int64_t s = forward->elem_size;
    int64_t algo = 0;
    int launches = 0;
    for (int k = 0; k < npart && rc == GBX_SUCCESS; k++) {
        const int64_t n = plan.elem_off[k + 1] - plan.elem_off[k];
        if (n == 0) { req->parts.push_back(nullptr); continue; }
        gbx_request_s *c = new_request(o, stream);
        req->parts.push_back(c);
        if (!c->done) { rc = GBX_ERR_CUDA; break; }
        c->kind = 0;
        c->graph = forward->graph;
        c->src = forward->src;
        c->dst = forward->dst;
        c->src_bytes = forward->src_bytes;
        c->dst_bytes = forward->dst_bytes;
        c->elem_size = s;
        c->dtype = forward->dtype;
        c->align = forward->align;
        c->algorithm = GBX_ALG_STANDARD;
        const int64_t ns = plan.seg_off[k + 1] - plan.seg_off[k];
        rc = gbx_make_copy_op(c, 0, c->src, ROLE_SRC, c->dst, ROLE_DST, plan.segs + plan.seg_off[k], ns,
                              plan.idx + plan.elem_off[k], n, n, 2 * n * s + 4 * n + ns * (int64_t)sizeof(Seg));
        if (rc == GBX_SUCCESS) rc = finalize(c);
        if (rc == GBX_SUCCESS) {
            c->info.V = n;
            c->info.elem_size = s;
            c->info.user_bytes = 2 * n * s;
            algo += c->info.algo_bytes;
            launches += c->info.launches;
        }
    }
    for (int k = 0; k < npart && rc == GBX_SUCCESS; k++) {
        cudaEvent_t ev;
        if (gbx_event_create(&ev) != cudaSuccess) { rc = GBX_ERR_CUDA; break; }
        req->part_ev.push_back(ev);
    }
    if (rc != GBX_SUCCESS) {
        req->part_ready.assign(req->part_ev.size(), 0);
        destroy_request(req);
        return rc;
    }
    req->feed = plan.feed;
    gbx_request_info_t &I = req->info;
    I = forward->info;
    I.kind = 2;
    I.levels = 1;
    I.launches = launches;
    I.algo_bytes = algo;
    *request = req;
    return GBX_SUCCESS;
}

extern "C" int gbx_pready(gbx_request_t req, int p, void *stream) {
    if (!req || req->kind != 2 || p < 0 || p >= req->npart) return GBX_ERR_ARG;
    GbxRange range("gbx.pready");
    if (!req->active || req->part_ready[p]) return GBX_ERR_STATE;
    cudaStream_t st = stream ? (cudaStream_t)stream : req->stream;
    gbx_request_s *c = req->parts[p];
    if (c) {
        if (c->use_graph && c->exec) GBX_CUDA_TRY(cudaGraphLaunch(c->exec, st));
        else GBX_CUDA_TRY(enqueue_levels(c->launches, st));
    }
    GBX_CUDA_TRY(cudaEventRecord(req->part_ev[p], st));
    req->part_ready[p] = 1;
    req->nready++;
    return GBX_SUCCESS;
}

static bool feeds(const gbx_request_s *req, int j, int k) {
    const int words = (req->npart + 31) / 32;
    return (req->feed[(size_t)j * words + (k >> 5)] >> (k & 31)) & 1u;
}

extern "C" int gbx_parrived(gbx_request_t req, int j, int *flag) {
    if (!req || req->kind != 2 || j < 0 || j >= req->nrpart || !flag) return GBX_ERR_ARG;
    if (!req->active) return GBX_ERR_STATE;
    *flag = 1;
    for (int k = 0; k < req->npart; k++) {
        if (!feeds(req, j, k)) continue;
        if (!req->part_ready[k]) { *flag = 0; return GBX_SUCCESS; }
        cudaError_t e = cudaEventQuery(req->part_ev[k]);
        if (e == cudaErrorNotReady) { *flag = 0; return GBX_SUCCESS; }
        if (e != cudaSuccess) {
            gbx_note_cuda_error(e, "event query", __FILE__, __LINE__);
            return GBX_ERR_CUDA;
        }
    }
    return GBX_SUCCESS;
}

extern "C" int gbx_parrived_stream(gbx_request_t req, int j, void *stream) {
    if (!req || req->kind != 2 || j < 0 || j >= req->nrpart) return GBX_ERR_ARG;
    if (!req->active) return GBX_ERR_STATE;
    for (int k = 0; k < req->npart; k++)
        if (feeds(req, j, k) && !req->part_ready[k]) return GBX_ERR_STATE;
    for (int k = 0; k < req->npart; k++)
        if (feeds(req, j, k)) GBX_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, req->part_ev[k], 0));
    return GBX_SUCCESS;
}

extern "C" int gbx_backward_init(gbx_request_t forward, const void *grad_recv, void *grad_send, int accumulate,
                                 const char *info, void *stream, gbx_request_t *request) {
    if (!request) return GBX_ERR_ARG;
    *request = nullptr;
    if (!forward || forward->kind != 0) return GBX_ERR_ARG;
    if (forward->dtype != GBX_F32 && forward->dtype != GBX_F64) return GBX_ERR_ARG;
    const int dsz = forward->dtype == GBX_F64 ? 8 : 4;
    if (forward->elem_size % dsz) return GBX_ERR_ARG;
    if ((forward->dst_bytes > 0 && !grad_recv) || (forward->src_bytes > 0 && !grad_send)) return GBX_ERR_ARG;
    GBX_TRY(gbx_check_data_buf(grad_recv, forward->dst_bytes));
    GBX_TRY(gbx_check_data_buf(grad_send, forward->src_bytes));
    Opts o = parse_info(info);
    if (!o.ok) return GBX_ERR_ARG;
    GbxRange range("gbx.setup.backward");
    gbx_request_s *req = new_request(o, stream);
    if (!req->done) { destroy_request(req); return GBX_ERR_CUDA; }
    req->kind = 1;
    req->forward = forward;
    req->graph = forward->graph;
    req->src = (const char *)grad_recv;
    req->dst = (char *)grad_send;
    req->src_bytes = forward->dst_bytes;
    req->dst_bytes = forward->src_bytes;
    req->elem_size = forward->elem_size;
    req->dtype = forward->dtype;
    req->algorithm = forward->algorithm;
    req->align = forward->align | (uint64_t)(uintptr_t)grad_recv | (uint64_t)(uintptr_t)grad_send;
    int rc = gbx_setup_backward(req, accumulate ? 1 : 0);
    if (rc == GBX_SUCCESS) rc = finalize(req);
    if (rc != GBX_SUCCESS) { destroy_request(req); return rc; }
    *request = req;
    return GBX_SUCCESS;
}

// ------------------------------------------------------------- start / wait
static int enqueue_start(gbx_request_s *req) {
    GbxRange range(req->kind == 1 ? "gbx.start.backward"
                   : req->algorithm == GBX_ALG_LOCALITY ? "gbx.start.locality" : "gbx.start.standard");
    // the exchange overwrites the bound destination: it follows the last host read-back of it
    if (req->host_down_pending) GBX_CUDA_TRY(cudaStreamWaitEvent(req->stream, req->host_down_ev, 0));
    if (req->use_graph && req->exec) {
        GBX_CUDA_TRY(cudaGraphLaunch(req->exec, req->stream));
    } else {
        GBX_CUDA_TRY(enqueue_levels(req->launches, req->stream));
    }
    GBX_CUDA_TRY(cudaEventRecord(req->done, req->stream));
    req->pending = nullptr;
    req->active = 1;
    return GBX_SUCCESS;
}

extern "C" int gbx_start(gbx_request_t req) {
    if (!req) return GBX_ERR_ARG;
    if (req->active) return GBX_ERR_ACTIVE;
    if (req->kind == 2) {   // partitioned: open an epoch; data moves at gbx_pready
        std::fill(req->part_ready.begin(), req->part_ready.end(), 0);
        req->nready = 0;
        req->active = 1;
        return GBX_SUCCESS;
    }
    return enqueue_start(req);
}

static cudaEvent_t pending_event(gbx_request_s *req) { return req->pending ? *req->pending : req->done; }

// partitioned: 1 when every marked partition's moves are done (0 if still running)
static int parts_done(gbx_request_s *req, int *flag) {
    *flag = 1;
    for (int k = 0; k < req->npart; k++) {
        if (!req->part_ready[k]) continue;
        cudaError_t e = cudaEventQuery(req->part_ev[k]);
        if (e == cudaErrorNotReady) { *flag = 0; return GBX_SUCCESS; }
        if (e != cudaSuccess) {
            gbx_note_cuda_error(e, "event query", __FILE__, __LINE__);
            return GBX_ERR_CUDA;
        }
    }
    return GBX_SUCCESS;
}

// Reads and clears the request's status word once its kernels have finished:
// GBX_ERR_DEVICE_WAIT when one of them gave up a bounded wait or skipped a bad piece.
static int take_status(gbx_request_s *req) {
    volatile int *w = req->status_host;
    if (!w || *w == 0) return GBX_SUCCESS;
    *w = 0;
    return GBX_ERR_DEVICE_WAIT;
}

extern "C" int gbx_test(gbx_request_t req, int *flag) {
    if (!req || !flag) return GBX_ERR_ARG;
    *flag = 1;
    if (!req->active) return take_status(req);   // e.g. completed by gbx_wait_stream
    if (req->kind == 2) {
        if (req->nready < req->npart) { *flag = 0; return GBX_ERR_STATE; }
        GBX_TRY(parts_done(req, flag));
        if (!*flag) return GBX_SUCCESS;
        req->active = 0;
        int rc = GBX_SUCCESS;
        for (gbx_request_s *c : req->parts)
            if (c && take_status(c) != GBX_SUCCESS) rc = GBX_ERR_DEVICE_WAIT;
        return rc;
    }
    cudaError_t e = cudaEventQuery(pending_event(req));
    if (e == cudaErrorNotReady) { *flag = 0; return GBX_SUCCESS; }
    if (e != cudaSuccess) {
        gbx_note_cuda_error(e, "event query", __FILE__, __LINE__);
        return GBX_ERR_CUDA;
    }
    req->active = 0;
    req->pending = nullptr;
    return take_status(req);
}

#define GBX_WAIT_SPIN_MS 20.0

extern "C" int gbx_wait(gbx_request_t req) {
    if (!req) return GBX_ERR_ARG;
    if (!req->active) return take_status(req);
    // polls (yielding the core) for the first GBX_WAIT_SPIN_MS, then sleeps between polls: a
    // sleeping thread wakes tens of microseconds after the work ends (the kernel's timer
    // slack), which would show in every start + wait of a millisecond-long exchange
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int flag = 0;
        const int rc = gbx_test(req, &flag);
        if (rc != GBX_SUCCESS || flag) return rc;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > req->timeout_ms) return GBX_ERR_TIMEOUT;
        if (ms > GBX_WAIT_SPIN_MS) std::this_thread::sleep_for(std::chrono::microseconds(20));
        else std::this_thread::yield();
    }
}

extern "C" int gbx_wait_stream(gbx_request_t req, void *stream) {
    if (!req) return GBX_ERR_ARG;
    if (!req->active) return GBX_SUCCESS;
    if (req->kind == 2) {
        if (req->nready < req->npart) return GBX_ERR_STATE;
        for (int k = 0; k < req->npart; k++)
            GBX_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, req->part_ev[k], 0));
        req->active = 0;
        return GBX_SUCCESS;
    }
    GBX_CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)stream, pending_event(req), 0));
    req->active = 0;
    req->pending = nullptr;
    return GBX_SUCCESS;
}

// Waits for every request (each one is completed even when an earlier one reports an
// error); returns the first error, in request order.
extern "C" int gbx_waitall(int count, gbx_request_t *reqs) {
    if (count < 0 || (count > 0 && !reqs)) return GBX_ERR_ARG;
    int first = GBX_SUCCESS;
    for (int i = 0; i < count; i++) {
        const int rc = gbx_wait(reqs[i]);
        if (rc != GBX_SUCCESS && first == GBX_SUCCESS) first = rc;
    }
    return first;
}

// A batch pools copies by vector width.  An op whose own tuning kept a narrower vector than its
// alignment allows (common for small ops, whose timings are noise) would add a launch of its own;
// in a batch it runs at its widest vector instead, through a batch-owned descriptor (same
// elements, same bytes, its own tile table), so that it joins its dtype's main launch.
static int widen_candidate(const HostOp &op) {
    const uintptr_t a = (uintptr_t)op.cd.src | (uintptr_t)op.cd.dst | (uintptr_t)op.cd.src2;
    return op.kind == 0 && op.flat_ok && op.cd.flat != 8 && op.cd.flat != 9 && op.cd.vec < op.max_vec &&
           op.max_vec >= 4 && (a & (uintptr_t)(op.max_vec - 1)) == 0;
}

static int widen_op(DevPool &mem, HostOp &c, int64_t s, cudaStream_t st) {
    const int vec = c.max_vec, cpe = (int)(s / vec);
    int shift = -1;
    if ((cpe & (cpe - 1)) == 0) { shift = 0; while ((1 << shift) < cpe) shift++; }
    CopyDesc &d = c.cd;
    d.vec = vec; d.cpe = cpe; d.cpe_shift = shift;
    d.cpe_magic = shift >= 0 ? 0u : (uint32_t)(((1ull << 32) + (uint64_t)cpe - 1) / (uint64_t)cpe);
    d.nchunks = d.nelem * cpe;
    d.ntiles = ceil_div(d.nchunks, GBX_TILE);
    // segment and pipelined forms run as the plain flat form the op also has (stream forms stay)
    if (d.flat < 10) d.flat = (d.flat & 3) == 3 ? 3 : 1;
    GBX_TRY(mem.get(&c.d_tile_e0, d.ntiles + 1));
    d.tile_e0 = c.d_tile_e0;
    d.tile_seg = nullptr;
    GBX_TRY(gbx_build_tile_meta(nullptr, 0, cpe, d.ntiles, nullptr, c.d_tile_e0, st));
    GBX_TRY(mem.alloc(&c.d_desc, sizeof(CopyDesc)));
    GBX_CUDA_TRY(cudaMemcpyAsync(c.d_desc, &d, sizeof(CopyDesc), cudaMemcpyHostToDevice, st));
    return GBX_SUCCESS;
}

extern "C" int gbx_startall(int count, gbx_request_t *reqs) {
    if (count <= 0 || !reqs) return GBX_ERR_ARG;
    GbxRange range("gbx.startall");
    for (int i = 0; i < count; i++) {
        if (!reqs[i]) return GBX_ERR_ARG;
        if (reqs[i]->kind == 2) return GBX_ERR_UNSUPPORTED;
        if (reqs[i]->active) return GBX_ERR_ACTIVE;
        for (int j = 0; j < i; j++) if (reqs[j] == reqs[i]) return GBX_ERR_ARG;
    }
    for (int i = 0; i < count; i++)   // destinations still being read back to the host
        if (reqs[i]->host_down_pending) GBX_CUDA_TRY(cudaStreamWaitEvent(reqs[0]->stream, reqs[i]->host_down_ev, 0));
    std::vector<gbx_request_s *> key(reqs, reqs + count);
    Batch *b = nullptr;
    for (Batch *c : reqs[0]->batches)
        if (c->members == key) { b = c; break; }
    if (!b) {
        b = new Batch();
        b->members = key;
        cudaStream_t st = reqs[0]->stream;
        std::vector<HostOp *> ops;
        std::vector<int> dts;
        int rc0 = GBX_SUCCESS;
        size_t nwide = 0;
        for (gbx_request_s *r : key)
            for (HostOp &op : r->ops) nwide += widen_candidate(op);
        b->widened.reserve(nwide);   // stable addresses for the pointers below
        for (gbx_request_s *r : key)
            for (HostOp &op : r->ops) {
                HostOp *use = &op;
                if (rc0 == GBX_SUCCESS && widen_candidate(op)) {
                    b->widened.push_back(op);
                    b->widened_of.emplace_back(r, (size_t)(&op - r->ops.data()));
                    rc0 = widen_op(b->mem, b->widened.back(), r->elem_size, st);
                    use = &b->widened.back();
                }
                ops.push_back(use);
                dts.push_back(r->dtype);
            }
        if (rc0 != GBX_SUCCESS) {
            delete b;
            return rc0;
        }
        int tune = 1, cap = 0;
        for (gbx_request_s *r : key) {
            tune &= r->autotune && !r->forced_block;
            if (r->max_ctas > 0) cap = cap > 0 ? std::min(cap, r->max_ctas) : r->max_ctas;
        }
        int rc = build_levels(b->mem, ops, dts, b->launches, 1, st, tune, cap);
        if (rc == GBX_SUCCESS && gbx_event_create(&b->done) != cudaSuccess)
            rc = GBX_ERR_CUDA;
        if (rc == GBX_SUCCESS && !b->launches.empty()) rc = capture(b->launches, &b->exec);
        if (rc != GBX_SUCCESS) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->done) cudaEventDestroy(b->done);
            delete b;
            return rc;
        }
        for (gbx_request_s *r : key) r->batches.push_back(b);
    }
    cudaStream_t st = reqs[0]->stream;
    if (b->exec) GBX_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    GBX_CUDA_TRY(cudaEventRecord(b->done, st));
    for (gbx_request_s *r : key) {
        r->active = 1;
        r->pending = &b->done;
    }
    return GBX_SUCCESS;
}

// ---------------------------------------------------------------- re-binding
extern "C" int gbx_request_bind(gbx_request_t req, const void *src, void *dst) {
    if (!req) return GBX_ERR_ARG;
    if (req->active) return GBX_ERR_ACTIVE;
    if (req->kind == 2) {
        for (gbx_request_s *c : req->parts)
            if (c) GBX_TRY(gbx_request_bind(c, src, dst));
        if (src) req->src = (const char *)src;
        if (dst) req->dst = (char *)dst;
        return GBX_SUCCESS;
    }
    GBX_TRY(gbx_check_data_buf(src, req->src_bytes));
    GBX_TRY(gbx_check_data_buf(dst, req->dst_bytes));
    const char *ns = src ? (const char *)src : req->src;
    char *nd = dst ? (char *)dst : req->dst;
    const bool ns_host = src && host_mem(src), nd_host = dst && host_mem(dst);
    for (HostOp &op : req->ops) {
        const int vec = op.kind == 0 ? op.cd.vec : op.fd.vec;
        if (((uintptr_t)ns & (uintptr_t)(vec - 1)) || ((uintptr_t)nd & (uintptr_t)(vec - 1))) return GBX_ERR_ARG;
        // an op tuned to a bulk-copy form cannot move to host memory
        if (op.kind == 0 && (op.cd.flat == 8 || op.cd.flat == 9) &&
            ((ns_host && op.cd.src_role == ROLE_SRC) || (nd_host && op.cd.dst_role == ROLE_DST)))
            return GBX_ERR_UNSUPPORTED;
    }
    for (HostOp &op : req->ops) {
        if (op.kind == 0) {
            if (op.cd.src_role == ROLE_SRC) op.cd.src = ns;
            if (op.cd.dst_role == ROLE_DST) op.cd.dst = nd;
        } else {
            if (op.fd.out_role == ROLE_DST) op.fd.out = nd;
            if (op.fd.a_role == ROLE_SRC) op.fd.bufA = ns;
        }
        GBX_TRY(upload_desc(req, op));
    }
    req->src = ns;
    req->dst = nd;
    // cached batches hold their own widened copies of some of these ops: they follow the new
    // buffers, and a batch whose copy the new buffers no longer align is rebuilt at the next
    // gbx_startall
    std::vector<Batch *> stale;
    for (Batch *b : req->batches)
        for (size_t k = 0; k < b->widened.size(); k++) {
            if (b->widened_of[k].first != req) continue;
            const HostOp &o = req->ops[b->widened_of[k].second];
            HostOp &c = b->widened[k];
            c.cd.src = o.cd.src;
            c.cd.dst = o.cd.dst;
            if (((uintptr_t)c.cd.src | (uintptr_t)c.cd.dst) & (uintptr_t)(c.cd.vec - 1)) {
                stale.push_back(b);
                break;
            }
            GBX_CUDA_TRY(cudaMemcpyAsync(c.d_desc, &c.cd, sizeof(CopyDesc), cudaMemcpyHostToDevice, req->stream));
        }
    // a batch may run on another request's stream: its next start must see the new descriptors
    const bool batched = !req->batches.empty();
    for (Batch *b : stale) destroy_batch(b);
    if (batched) GBX_CUDA_TRY(cudaStreamSynchronize(req->stream));
    return GBX_SUCCESS;
}

static int host_streams(gbx_request_s *req) {
    if (req->host_up) return GBX_SUCCESS;
    GBX_CUDA_TRY(cudaStreamCreateWithFlags(&req->host_up, cudaStreamNonBlocking));
    GBX_CUDA_TRY(cudaStreamCreateWithFlags(&req->host_down, cudaStreamNonBlocking));
    GBX_CUDA_TRY(gbx_event_create(&req->host_up_ev));
    GBX_CUDA_TRY(gbx_event_create(&req->host_down_ev));
    GBX_CUDA_TRY(gbx_event_create(&req->host_mark));
    return GBX_SUCCESS;
}

extern "C" int gbx_start_host_async(gbx_request_t req, const void *host_src, void *host_dst) {
    if (!req) return GBX_ERR_ARG;
    if (req->kind == 2) return GBX_ERR_UNSUPPORTED;
    if (req->active) return GBX_ERR_ACTIVE;
    GBX_TRY(host_streams(req));
    if (host_src && req->src_bytes > 0) {
        // the upload overwrites the bound source: it follows everything already queued on the
        // request's stream (earlier exchanges that read the source)
        GBX_CUDA_TRY(cudaEventRecord(req->host_mark, req->stream));
        GBX_CUDA_TRY(cudaStreamWaitEvent(req->host_up, req->host_mark, 0));
        GBX_CUDA_TRY(cudaMemcpyAsync((void *)req->src, host_src, req->src_bytes, cudaMemcpyDefault,
                                     req->host_up));
        GBX_CUDA_TRY(cudaEventRecord(req->host_up_ev, req->host_up));
        GBX_CUDA_TRY(cudaStreamWaitEvent(req->stream, req->host_up_ev, 0));
    }
    GBX_TRY(enqueue_start(req));
    if (host_dst && req->dst_bytes > 0) {
        GBX_CUDA_TRY(cudaStreamWaitEvent(req->host_down, req->done, 0));
        GBX_CUDA_TRY(cudaMemcpyAsync(host_dst, req->dst, req->dst_bytes, cudaMemcpyDefault, req->host_down));
        GBX_CUDA_TRY(cudaEventRecord(req->host_down_ev, req->host_down));
        GBX_CUDA_TRY(cudaEventRecord(req->done, req->host_down));   // complete once read back
        req->host_down_pending = 1;
    }
    return GBX_SUCCESS;
}

extern "C" int gbx_start_host(gbx_request_t req, const void *host_src, void *host_dst) {
    if (!req || (req->src_bytes > 0 && !host_src) || (req->dst_bytes > 0 && !host_dst)) return GBX_ERR_ARG;
    GBX_TRY(gbx_start_host_async(req, host_src, host_dst));
    return gbx_wait(req);
}

extern "C" int gbx_request_get_info(gbx_request_t req, gbx_request_info_t *info) {
    if (!req || !info) return GBX_ERR_ARG;
    req->info.device_bytes = req->mem.bytes;
    *info = req->info;
    return GBX_SUCCESS;
}

extern "C" int gbx_request_free(gbx_request_t *req) {
    if (!req) return GBX_ERR_ARG;
    destroy_request(*req);
    *req = nullptr;
    return GBX_SUCCESS;
}
