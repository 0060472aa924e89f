/*
 * oracle.c -- plain, slow, CPU-only oracle for the data movement of a persistent
 * neighbourhood all-to-all-v over an emulated distributed-graph communicator.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py load it.  The GPU library does not call
 * it, include it, or share any code, header, table or helper with it.
 *
 * Source: Bienz, Schafer, Skjellum, "MPI Advance: Open-Source Message Passing
 * Optimizations" (arXiv 2309.07337).
 *
 *  * Section 2.2, Listings 3 and 4: the operation is MPI_Neighbor_alltoallv on a
 *    communicator built by MPI_Dist_graph_create_adjacent, in its persistent form
 *    (init once, then start / wait).  The paper names the call without restating its
 *    meaning, so the meaning is the MPI standard's:
 *      - rank r sends to its j-th out-neighbour d the sendcounts[j] elements that start
 *        at element sdispls[j] of its send buffer;
 *      - rank d receives from its i-th in-neighbour recvcounts[i] elements, stored from
 *        element rdispls[i] of its receive buffer;
 *      - when r lists d several times (a multigraph), the t-th listing of d in r's
 *        out-list pairs with the t-th listing of r in d's in-list;
 *      - paired counts must be equal (otherwise MPI_ERR_TRUNCATE);
 *      - receive locations not covered by any block are left untouched.
 *    The "pack by send index list" extension reads send slot q of rank r from element
 *    send_idx[q] of r's region instead of element q.
 *  * Section 2.2, last paragraph: the locality-aware variant takes a unique global index
 *    for every value sent and received, so that one value crosses a given pair of nodes
 *    only once.  When the caller gives none, a value is named by its source element (its
 *    byte offset in the send buffer): distinct elements stay distinct, and an element
 *    sent to several ranks of one node still crosses that node pair once.
 *  * Section 1: locality-aware aggregation sends inter-node traffic as one aggregated
 *    message per pair of nodes.  The steps followed here (the paper cites but does not
 *    print them): intra-node blocks are copied directly; every inter-node value is
 *    gathered once into the send aggregate of its node pair (deduplicated by global
 *    index, ordered by representative rank then global index); each node pair's
 *    aggregate is copied as one block; the destination node redistributes every
 *    received value to each receive slot that names it.
 *  * Backward: the exchange is linear, so its adjoint is the transpose of the forward
 *    0/1 map: every source element receives the sum of the gradients of all receive
 *    slots that read it.  Two fixed summation orders are defined (see orc_backward).
 *
 * Element bytes are copied with memcpy, never converted.  Floating-point sums use plain
 * IEEE adds in the payload precision, left to right, no contraction (build with
 * -ffp-contract=off and without fast-math).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,       /* bad argument or missing required array                 */
    ORC_ERR_RANK = 2,      /* neighbour rank outside [0, P)                            */
    ORC_ERR_TRUNCATE = 3,  /* unmatched edge, or paired counts differ                  */
    ORC_ERR_INDEX = 4,     /* displacement, slot or element index out of range         */
    ORC_ERR_DUP = 5,       /* one global index carried by different bytes             */
    ORC_ERR_GIDX = 6,      /* receive global index differs from the matched send index */
    ORC_ERR_NOMEM = 10,
    ORC_ERR_UNSUPPORTED = 11, /* a derived displacement beyond the int32 range           */
    ORC_ERR_OVERLAP = 13   /* two receive blocks write the same bytes                  */
};
enum { ORC_BYTES = 0, ORC_F32 = 1, ORC_F64 = 2 };

/* All arrays are host arrays.  Per-rank arguments of the MPI call are concatenated
 * over ranks: in-edge arrays follow in_ptr, out-edge arrays follow out_ptr.  Byte
 * offsets locate every rank's region inside one send and one receive buffer. */
typedef struct {
    int P, ppn;
    const int *in_ptr, *sources;        /* in-lists:  CSR, P+1 / in_ptr[P]        */
    const int *out_ptr, *dests;         /* out-lists: CSR, P+1 / out_ptr[P]       */
    const int *sendcounts, *sdispls;    /* one per out-edge                       */
    const int *recvcounts, *rdispls;    /* one per in-edge                        */
    const int64_t *send_base;           /* P byte offsets into the send buffer    */
    const int64_t *recv_base;           /* P byte offsets into the receive buffer */
    const int64_t *send_slot_ptr;       /* P+1 or NULL: send-slot CSR             */
    const int *send_idx;                /* NULL or element index of each send slot */
    const int64_t *recv_slot_ptr;       /* P+1 or NULL: receive-slot CSR          */
    const int64_t *global_sidx;         /* NULL or global index of each send slot */
    const int64_t *global_ridx;         /* NULL or global index of each recv slot */
    int64_t elem_size, sendbuf_bytes, recvbuf_bytes;
} orc_pattern;

#define MIN_ERR(e, c) do { if ((c) != ORC_OK && ((e) == ORC_OK || (c) < (e))) (e) = (c); } while (0)

/* ---------------------------------------------------------------- matching --- */

typedef struct { int key; int64_t pos; } kp_t;

static int cmp_kp(const void *x, const void *y) {
    const kp_t *a = (const kp_t *)x, *b = (const kp_t *)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

static int check_csr(int P, const int *ptr) {
    if (ptr[0] != 0) return ORC_ERR_ARG;
    for (int r = 0; r < P; r++)
        if (ptr[r + 1] < ptr[r]) return ORC_ERR_ARG;
    return ORC_OK;
}

/* match[e] = in-edge paired with out-edge e under the multigraph rule of the MPI
 * standard (the t-th listing of d by r pairs with the t-th listing of r by d). */
int orc_match(const orc_pattern *pt, int64_t *match) {
    int P = pt->P;
    if (P <= 0 || !pt->in_ptr || !pt->out_ptr || !match) return ORC_ERR_ARG;
    if (check_csr(P, pt->in_ptr) || check_csr(P, pt->out_ptr)) return ORC_ERR_ARG;
    int64_t n_in = pt->in_ptr[P], n_out = pt->out_ptr[P];
    if ((n_in && !pt->sources) || (n_out && !pt->dests)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n_in; i++)
        if (pt->sources[i] < 0 || pt->sources[i] >= P) return ORC_ERR_RANK;
    for (int64_t e = 0; e < n_out; e++)
        if (pt->dests[e] < 0 || pt->dests[e] >= P) return ORC_ERR_RANK;
    if (n_in != n_out) return ORC_ERR_TRUNCATE;
    if (n_in == 0) return ORC_OK;

    kp_t *in_s = malloc(sizeof(kp_t) * n_in), *out_s = malloc(sizeof(kp_t) * n_out);
    if (!in_s || !out_s) { free(in_s); free(out_s); return ORC_ERR_NOMEM; }
    for (int d = 0; d < P; d++) {
        for (int64_t i = pt->in_ptr[d]; i < pt->in_ptr[d + 1]; i++) {
            in_s[i].key = pt->sources[i];
            in_s[i].pos = i;
        }
        qsort(in_s + pt->in_ptr[d], pt->in_ptr[d + 1] - pt->in_ptr[d], sizeof(kp_t), cmp_kp);
    }
    int err = ORC_OK;
    for (int r = 0; r < P && !err; r++) {
        int64_t lo = pt->out_ptr[r], hi = pt->out_ptr[r + 1];
        for (int64_t e = lo; e < hi; e++) { out_s[e].key = pt->dests[e]; out_s[e].pos = e; }
        qsort(out_s + lo, hi - lo, sizeof(kp_t), cmp_kp);
        int64_t run = lo;
        for (int64_t x = lo; x < hi; x++) {
            if (x > lo && out_s[x].key != out_s[x - 1].key) run = x;
            int64_t t = x - run;               /* occurrence number of d in r's list */
            int d = out_s[x].key;
            /* first listing of r in d's sorted in-list */
            int64_t a = pt->in_ptr[d], b = pt->in_ptr[d + 1];
            while (a < b) {
                int64_t m = a + (b - a) / 2;
                if (in_s[m].key < r) a = m + 1; else b = m;
            }
            int64_t want = a + t;
            if (want >= pt->in_ptr[d + 1] || in_s[want].key != r) { err = ORC_ERR_TRUNCATE; break; }
            match[out_s[x].pos] = in_s[want].pos;
        }
    }
    free(in_s);
    free(out_s);
    return err;
}

/* ------------------------------------------------------------- validation --- */

static int64_t slots_of(const int64_t *ptr, int r) { return ptr[r + 1] - ptr[r]; }

/* Element index (within rank r's region) read by send slot q of rank r. */
static int64_t send_elem(const orc_pattern *pt, int r, int64_t q) {
    if (pt->send_idx) return pt->send_idx[pt->send_slot_ptr[r] + q];
    return q;
}

typedef struct { int64_t lo, hi; } range_t;
static int cmp_range(const void *x, const void *y) {
    const range_t *a = (const range_t *)x, *b = (const range_t *)y;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    return (a->hi > b->hi) - (a->hi < b->hi);
}

/* Checks everything the exchange needs; returns the smallest error code found. */
static int check_pattern(const orc_pattern *pt, const int64_t *match) {
    int P = pt->P;
    int64_t s = pt->elem_size;
    if (s <= 0 || !pt->sendcounts || !pt->sdispls || !pt->recvcounts || !pt->rdispls ||
        !pt->send_base || !pt->recv_base)
        return ORC_ERR_ARG;
    if ((pt->send_idx || pt->global_sidx) && !pt->send_slot_ptr) return ORC_ERR_ARG;
    if (pt->global_ridx && (!pt->recv_slot_ptr || !pt->global_sidx)) return ORC_ERR_ARG;
    int err = ORC_OK;
    int64_t n_out = pt->out_ptr[P];
    range_t *rr = malloc(sizeof(range_t) * (n_out ? n_out : 1));
    if (!rr) return ORC_ERR_NOMEM;
    int64_t nr = 0;
    for (int r = 0; r < P; r++) {
        if (pt->send_base[r] < 0) MIN_ERR(err, ORC_ERR_INDEX);
        if (pt->recv_base[r] < 0) MIN_ERR(err, ORC_ERR_INDEX);
    }
    for (int r = 0; r < P; r++) {
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            int64_t i = match[e];
            int64_t cnt = pt->sendcounts[e];
            if (pt->recvcounts[i] != cnt || cnt < 0) { MIN_ERR(err, ORC_ERR_TRUNCATE); continue; }
            int64_t sd = pt->sdispls[e], rd = pt->rdispls[i];
            int ok = 1;
            /* send side */
            if (sd < 0) ok = 0;
            else if (pt->send_slot_ptr) {
                if (sd + cnt > slots_of(pt->send_slot_ptr, r)) ok = 0;
            }
            if (ok && pt->send_base[r] >= 0) {
                if (!pt->send_idx) {
                    if (pt->send_base[r] + (sd + cnt) * s > pt->sendbuf_bytes) ok = 0;
                } else {
                    for (int64_t k = 0; k < cnt; k++) {
                        int64_t el = send_elem(pt, r, sd + k);
                        if (el < 0 || pt->send_base[r] + (el + 1) * s > pt->sendbuf_bytes) { ok = 0; break; }
                    }
                }
            } else ok = 0;
            /* receive side */
            if (rd < 0) ok = 0;
            else if (pt->recv_slot_ptr && rd + cnt > slots_of(pt->recv_slot_ptr, d)) ok = 0;
            else if (pt->recv_base[d] < 0 || pt->recv_base[d] + (rd + cnt) * s > pt->recvbuf_bytes) ok = 0;
            if (!ok) { MIN_ERR(err, ORC_ERR_INDEX); continue; }
            if (pt->global_ridx) {
                for (int64_t k = 0; k < cnt; k++)
                    if (pt->global_ridx[pt->recv_slot_ptr[d] + rd + k] !=
                        pt->global_sidx[pt->send_slot_ptr[r] + sd + k]) {
                        MIN_ERR(err, ORC_ERR_GIDX);
                        break;
                    }
            }
            if (cnt > 0) {
                rr[nr].lo = pt->recv_base[d] + rd * s;
                rr[nr].hi = rr[nr].lo + cnt * s;
                nr++;
            }
        }
    }
    if (err == ORC_OK && nr > 1) {
        qsort(rr, nr, sizeof(range_t), cmp_range);
        for (int64_t x = 1; x < nr; x++)
            if (rr[x].lo < rr[x - 1].hi) { err = ORC_ERR_OVERLAP; break; }
    }
    free(rr);
    return err;
}

static int prepare(const orc_pattern *pt, int64_t **match_out) {
    if (!pt || pt->P <= 0 || pt->ppn <= 0 || !pt->in_ptr || !pt->out_ptr) return ORC_ERR_ARG;
    int64_t n = pt->out_ptr[pt->P] > 0 ? pt->out_ptr[pt->P] : 1;
    int64_t *match = malloc(sizeof(int64_t) * n);
    if (!match) return ORC_ERR_NOMEM;
    int err = orc_match(pt, match);
    if (!err) err = check_pattern(pt, match);
    if (err) { free(match); return err; }
    *match_out = match;
    return ORC_OK;
}

/* Returns ORC_OK when the pattern is a valid exchange (used by the error-path tests). */
int orc_validate(const orc_pattern *pt) {
    int64_t *match = NULL;
    int err = prepare(pt, &match);
    free(match);
    return err;
}

/* ------------------------------------------------------ standard exchange --- */

/* The definition: for every out-edge e of rank r to d, paired with in-edge i of d,
 *   recv[d][rdispls[i] + k] = send[r][elem(sdispls[e] + k)],  0 <= k < sendcounts[e]. */
int orc_standard(const orc_pattern *pt, const uint8_t *sendbuf, uint8_t *recvbuf) {
    int64_t *match = NULL;
    int err = prepare(pt, &match);
    if (err) return err;
    int64_t s = pt->elem_size;
    for (int r = 0; r < pt->P; r++) {
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            int64_t i = match[e];
            for (int64_t k = 0; k < pt->sendcounts[e]; k++) {
                int64_t src = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                int64_t dst = pt->recv_base[d] + (pt->rdispls[i] + k) * s;
                memcpy(recvbuf + dst, sendbuf + src, (size_t)s);
            }
        }
    }
    free(match);
    return ORC_OK;
}

/* ------------------------------------------------ locality-aware exchange --- */

static int node_of(const orc_pattern *pt, int r) { return r / pt->ppn; }
static int node_size(const orc_pattern *pt, int a) {
    int n = pt->P - a * pt->ppn;
    return n < pt->ppn ? n : pt->ppn;
}
/* Leader ranks of node pair (a, b): the rank of node a that owns the send aggregate
 * and the rank of node b that owns the receive aggregate (spread over the node). */
static int send_leader(const orc_pattern *pt, int a, int b) { return a * pt->ppn + b % node_size(pt, a); }
static int recv_leader(const orc_pattern *pt, int a, int b) { return b * pt->ppn + a % node_size(pt, b); }

typedef struct {
    int64_t gidx;
    int a, b, r, d;
    int64_t e, k;      /* out-edge and position: the order that picks a representative */
    int64_t src_off;   /* byte offset of the source element in the send buffer          */
    int64_t p;         /* receive slot position within d's receive view                 */
    int64_t recv_off;  /* byte offset of the receive element                            */
    int64_t t;         /* rank of its (a, b, gidx) value among distinct values          */
} xrec_t;

typedef struct {
    int a, b, rep_r;
    int64_t gidx, rep_src_off, t;
} uval_t;

static int cmp_xrec_value(const void *x, const void *y) {
    const xrec_t *p = (const xrec_t *)x, *q = (const xrec_t *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->gidx != q->gidx) return p->gidx < q->gidx ? -1 : 1;
    if (p->e != q->e) return p->e < q->e ? -1 : 1;
    return (p->k > q->k) - (p->k < q->k);
}

static int cmp_uval_order(const void *x, const void *y) {
    const uval_t *p = (const uval_t *)x, *q = (const uval_t *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->rep_r != q->rep_r) return p->rep_r < q->rep_r ? -1 : 1;
    return (p->gidx > q->gidx) - (p->gidx < q->gidx);
}

typedef struct {
    int64_t *match;
    xrec_t *x;        /* inter-node elements, sorted by (a, b, gidx, e, k)        */
    int64_t nx;
    uval_t *u;        /* distinct values in aggregate order (a, b, rep_r, gidx)   */
    int64_t nu;
    int64_t *pos_of_t;/* aggregate position of the t-th distinct value            */
    int64_t stats[16];
} loc_t;

static void loc_free(loc_t *L) {
    free(L->match); free(L->x); free(L->u); free(L->pos_of_t);
    memset(L, 0, sizeof(*L));
}

/* Builds the deduplicated aggregate layout and the statistics. */
static int loc_build(const orc_pattern *pt, const uint8_t *sendbuf, loc_t *L) {
    memset(L, 0, sizeof(*L));
    if (!pt) return ORC_ERR_ARG;
    int err = prepare(pt, &L->match);
    if (err) return err;
    int64_t s = pt->elem_size;
    int64_t V = 0, E = pt->out_ptr[pt->P], Enz = 0, Vd = 0, Vx = 0, Mx = 0, Md = 0;
    for (int r = 0; r < pt->P; r++)
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int64_t c = pt->sendcounts[e];
            V += c;
            if (c > 0) Enz++;
            if (node_of(pt, r) == node_of(pt, pt->dests[e])) { Vd += c; if (c > 0) Md++; }
            else { Vx += c; if (c > 0) Mx++; }
        }
    L->x = malloc(sizeof(xrec_t) * (Vx ? Vx : 1));
    if (!L->x) { loc_free(L); return ORC_ERR_NOMEM; }
    int64_t n = 0;
    for (int r = 0; r < pt->P; r++)
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            if (node_of(pt, r) == node_of(pt, d)) continue;
            int64_t i = L->match[e];
            for (int64_t k = 0; k < pt->sendcounts[e]; k++) {
                xrec_t *x = &L->x[n++];
                int64_t q = pt->sdispls[e] + k;
                x->src_off = pt->send_base[r] + send_elem(pt, r, q) * s;
                /* without global indices a value is named by its source element */
                x->gidx = pt->global_sidx ? pt->global_sidx[pt->send_slot_ptr[r] + q] : x->src_off;
                x->a = node_of(pt, r); x->b = node_of(pt, d); x->r = r; x->d = d;
                x->e = e; x->k = k;
                x->p = pt->rdispls[i] + k;
                x->recv_off = pt->recv_base[d] + x->p * s;
            }
        }
    L->nx = n;
    qsort(L->x, n, sizeof(xrec_t), cmp_xrec_value);
    /* distinct (a, b, gidx); the first occurrence in (e, k) order is the representative */
    int64_t nu = 0;
    for (int64_t j = 0; j < n; j++)
        if (j == 0 || L->x[j].a != L->x[j - 1].a || L->x[j].b != L->x[j - 1].b ||
            L->x[j].gidx != L->x[j - 1].gidx)
            nu++;
    L->u = malloc(sizeof(uval_t) * (nu ? nu : 1));
    L->pos_of_t = malloc(sizeof(int64_t) * (nu ? nu : 1));
    if (!L->u || !L->pos_of_t) { loc_free(L); return ORC_ERR_NOMEM; }
    int64_t t = -1;
    for (int64_t j = 0; j < n; j++) {
        xrec_t *x = &L->x[j];
        int fresh = (j == 0) || x->a != L->x[j - 1].a || x->b != L->x[j - 1].b || x->gidx != L->x[j - 1].gidx;
        if (fresh) {
            t++;
            L->u[t].a = x->a; L->u[t].b = x->b; L->u[t].gidx = x->gidx;
            L->u[t].rep_r = x->r; L->u[t].rep_src_off = x->src_off; L->u[t].t = t;
        } else if (sendbuf && memcmp(sendbuf + x->src_off, sendbuf + L->u[t].rep_src_off, (size_t)s) != 0) {
            err = ORC_ERR_DUP;
        }
        x->t = t;
    }
    L->nu = nu;
    if (err) { loc_free(L); return err; }
    qsort(L->u, nu, sizeof(uval_t), cmp_uval_order);
    for (int64_t q = 0; q < nu; q++) L->pos_of_t[L->u[q].t] = q;

    /* statistics */
    int64_t pairs = 0, m1 = 0, m3 = 0;
    for (int64_t q = 0; q < nu; q++) {
        uval_t *v = &L->u[q];
        int new_pair = q == 0 || v->a != L->u[q - 1].a || v->b != L->u[q - 1].b;
        if (new_pair) pairs++;
        if (new_pair || v->rep_r != L->u[q - 1].rep_r)
            if (v->rep_r != send_leader(pt, v->a, v->b)) m1++;
    }
    /* distinct (a, d) receiving inter-node traffic, d not the receive leader */
    {
        int nn = (pt->P + pt->ppn - 1) / pt->ppn;
        unsigned char *seen = calloc((size_t)nn * (size_t)pt->P, 1);
        if (!seen) { loc_free(L); return ORC_ERR_NOMEM; }
        for (int64_t j = 0; j < n; j++) {
            xrec_t *x = &L->x[j];
            size_t key = (size_t)x->a * (size_t)pt->P + (size_t)x->d;
            if (!seen[key]) {
                seen[key] = 1;
                if (x->d != recv_leader(pt, x->a, x->b)) m3++;
            }
        }
        free(seen);
    }
    L->stats[0] = V;   L->stats[1] = E;   L->stats[2] = Enz;
    L->stats[3] = Vd;  L->stats[4] = Vx;  L->stats[5] = nu;
    L->stats[6] = pairs; L->stats[7] = Mx; L->stats[8] = Md;
    L->stats[9] = m1;  L->stats[10] = m3;
    return ORC_OK;
}

/* Statistics of the locality-aware form without moving data:
 *  [0] V elements, [1] E edges, [2] edges with data, [3] intra-node elements,
 *  [4] inter-node elements, [5] distinct inter-node values (= step 1 and step 2 volume),
 *  [6] node pairs with traffic (= step 2 messages), [7] inter-node messages of the
 *  standard form, [8] intra-node messages of the standard form, [9] step 1 messages
 *  (a rank sending to a different send leader), [10] step 3 messages (a receive leader
 *  sending to a different rank). */
int orc_locality_stats(const orc_pattern *pt, int64_t *stats) {
    loc_t L;
    int err = loc_build(pt, NULL, &L);
    if (err) return err;
    memcpy(stats, L.stats, sizeof(L.stats));
    loc_free(&L);
    return ORC_OK;
}

/* Aggregate layout export for map tests: for each aggregate position q, its node pair,
 * global index and representative rank. Arrays are sized by orc_locality_stats()[5]. */
int orc_locality_layout(const orc_pattern *pt, int *a, int *b, int64_t *gidx, int *rep_r) {
    loc_t L;
    int err = loc_build(pt, NULL, &L);
    if (err) return err;
    for (int64_t q = 0; q < L.nu; q++) {
        a[q] = L.u[q].a; b[q] = L.u[q].b; gidx[q] = L.u[q].gidx; rep_r[q] = L.u[q].rep_r;
    }
    loc_free(&L);
    return ORC_OK;
}

/* Three-step locality-aware exchange.  Also returns the statistics (may be NULL). */
int orc_locality(const orc_pattern *pt, const uint8_t *sendbuf, uint8_t *recvbuf, int64_t *stats) {
    loc_t L;
    int err = loc_build(pt, sendbuf, &L);
    if (err) return err;
    int64_t s = pt->elem_size;
    uint8_t *S = malloc((size_t)(L.nu ? L.nu : 1) * (size_t)s);
    uint8_t *R = malloc((size_t)(L.nu ? L.nu : 1) * (size_t)s);
    if (!S || !R) { free(S); free(R); loc_free(&L); return ORC_ERR_NOMEM; }
    /* step 0: intra-node blocks go directly */
    for (int r = 0; r < pt->P; r++)
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            if (node_of(pt, r) != node_of(pt, d)) continue;
            int64_t i = L.match[e];
            for (int64_t k = 0; k < pt->sendcounts[e]; k++) {
                int64_t src = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                int64_t dst = pt->recv_base[d] + (pt->rdispls[i] + k) * s;
                memcpy(recvbuf + dst, sendbuf + src, (size_t)s);
            }
        }
    /* step 1: every distinct value is written once into its node pair's send aggregate */
    for (int64_t q = 0; q < L.nu; q++)
        memcpy(S + q * s, sendbuf + L.u[q].rep_src_off, (size_t)s);
    /* step 2: one block per node pair, send aggregate -> receive aggregate */
    for (int64_t q0 = 0; q0 < L.nu;) {
        int64_t q1 = q0;
        while (q1 < L.nu && L.u[q1].a == L.u[q0].a && L.u[q1].b == L.u[q0].b) q1++;
        memcpy(R + q0 * s, S + q0 * s, (size_t)((q1 - q0) * s));
        q0 = q1;
    }
    /* step 3: the receiving node hands every value to each receive slot that names it */
    for (int64_t j = 0; j < L.nx; j++) {
        xrec_t *x = &L.x[j];
        memcpy(recvbuf + x->recv_off, R + L.pos_of_t[x->t] * s, (size_t)s);
    }
    if (stats) memcpy(stats, L.stats, sizeof(L.stats));
    free(S); free(R);
    loc_free(&L);
    return ORC_OK;
}

/* --------------------------------------------------------------- backward --- */

/* One additive term of a source element's gradient. */
typedef struct {
    int64_t row;      /* byte offset of the source element (its identity)          */
    int64_t group;    /* destination node (node-blocked order) or 0 (standard)     */
    int64_t o1, o2;   /* order inside the group                                    */
    const uint8_t *val;
} term_t;

static int cmp_term(const void *x, const void *y) {
    const term_t *p = (const term_t *)x, *q = (const term_t *)y;
    if (p->row != q->row) return p->row < q->row ? -1 : 1;
    if (p->group != q->group) return p->group < q->group ? -1 : 1;
    if (p->o1 != q->o1) return p->o1 < q->o1 ? -1 : 1;
    return (p->o2 > q->o2) - (p->o2 < q->o2);
}

/* dst = a + b component-wise in the payload precision (memcpy keeps it alignment-safe). */
static void add_elem(int dtype, int64_t s, uint8_t *dst, const uint8_t *a, const uint8_t *b) {
    if (dtype == ORC_F64) {
        for (int64_t c = 0; c < s; c += 8) {
            double x, y, z;
            memcpy(&x, a + c, 8); memcpy(&y, b + c, 8);
            z = x + y;
            memcpy(dst + c, &z, 8);
        }
    } else {
        for (int64_t c = 0; c < s; c += 4) {
            float x, y, z;
            memcpy(&x, a + c, 4); memcpy(&y, b + c, 4);
            z = x + y;
            memcpy(dst + c, &z, 4);
        }
    }
}

/* Folds sorted terms row by row: inside a group, left to right; the group sums, left to
 * to right in group order; then either stores the result or adds it to the old value. */
static void fold_rows(const term_t *t, int64_t n, int dtype, int64_t s, int accumulate,
                      uint8_t *out, uint8_t *gacc, uint8_t *racc) {
    int64_t j = 0;
    while (j < n) {
        int64_t row = t[j].row;
        int have_row = 0;
        while (j < n && t[j].row == row) {
            int64_t g = t[j].group;
            memcpy(gacc, t[j].val, (size_t)s);
            j++;
            while (j < n && t[j].row == row && t[j].group == g) {
                add_elem(dtype, s, gacc, gacc, t[j].val);
                j++;
            }
            if (!have_row) { memcpy(racc, gacc, (size_t)s); have_row = 1; }
            else add_elem(dtype, s, racc, racc, gacc);
        }
        if (accumulate) add_elem(dtype, s, out + row, out + row, racc);
        else memcpy(out + row, racc, (size_t)s);
    }
}

/* Reverse exchange: grad_send[src] (+)= sum of grad_recv over the receive slots that read
 * src.  grad_recv has the receive buffer's layout, grad_send the send buffer's.
 * form 0 (standard order): one left-to-right sum per source element over its receive
 *   slots ordered by (destination rank, receive position).
 * form 1 (node-blocked order, the reverse of the three steps): per distinct inter-node
 *   value, the gradients of the slots that name it are summed in (destination rank,
 *   receive position) order (reverse step 3), copied back across the node pair (reverse
 *   step 2), and each source element folds its groups in ascending destination node:
 *   its own node's group holds its direct terms in (rank, position) order, a remote
 *   node's group holds the values it represents for that node in aggregate order.
 * accumulate = 0 stores the sum, 1 adds the sum to the existing value; elements that no
 * slot reads are left untouched either way. */
int orc_backward(const orc_pattern *pt, int form, int dtype, int accumulate,
                 const uint8_t *grad_recv, uint8_t *grad_send) {
    if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_ARG;
    int64_t s = pt->elem_size;
    int64_t dsz = dtype == ORC_F64 ? 8 : 4;
    if (s <= 0 || s % dsz) return ORC_ERR_ARG;
    uint8_t *gacc = malloc((size_t)s), *racc = malloc((size_t)s);
    if (!gacc || !racc) { free(gacc); free(racc); return ORC_ERR_NOMEM; }
    int err = ORC_OK;
    if (form == 0) {
        int64_t *match = NULL;
        err = prepare(pt, &match);
        if (err) { free(gacc); free(racc); return err; }
        int64_t V = 0;
        for (int64_t e = 0; e < pt->out_ptr[pt->P]; e++) V += pt->sendcounts[e];
        term_t *t = malloc(sizeof(term_t) * (V ? V : 1));
        if (!t) { free(match); free(gacc); free(racc); return ORC_ERR_NOMEM; }
        int64_t n = 0;
        for (int r = 0; r < pt->P; r++)
            for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
                int d = pt->dests[e];
                int64_t i = match[e];
                for (int64_t k = 0; k < pt->sendcounts[e]; k++) {
                    int64_t p = pt->rdispls[i] + k;
                    t[n].row = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                    t[n].group = 0;
                    t[n].o1 = d;
                    t[n].o2 = p;
                    t[n].val = grad_recv + pt->recv_base[d] + p * s;
                    n++;
                }
            }
        qsort(t, n, sizeof(term_t), cmp_term);
        fold_rows(t, n, dtype, s, accumulate, grad_send, gacc, racc);
        free(t);
        free(match);
    } else if (form == 1) {
        loc_t L;
        err = loc_build(pt, NULL, &L);
        if (err) { free(gacc); free(racc); return err; }
        /* reverse step 3: per distinct value, its receive slots in (d, p) order */
        uint8_t *gR = malloc((size_t)(L.nu ? L.nu : 1) * (size_t)s);
        uint8_t *gS = malloc((size_t)(L.nu ? L.nu : 1) * (size_t)s);
        term_t *t3 = malloc(sizeof(term_t) * (L.nx ? L.nx : 1));
        int64_t nterm = L.nu + L.stats[3];
        term_t *t1 = malloc(sizeof(term_t) * (nterm ? nterm : 1));
        if (!gR || !gS || !t3 || !t1) {
            free(gR); free(gS); free(t3); free(t1); loc_free(&L); free(gacc); free(racc);
            return ORC_ERR_NOMEM;
        }
        for (int64_t j = 0; j < L.nx; j++) {
            xrec_t *x = &L.x[j];
            t3[j].row = L.pos_of_t[x->t] * s;
            t3[j].group = 0;
            t3[j].o1 = x->d;
            t3[j].o2 = x->p;
            t3[j].val = grad_recv + x->recv_off;
        }
        qsort(t3, L.nx, sizeof(term_t), cmp_term);
        fold_rows(t3, L.nx, dtype, s, 0, gR, gacc, racc);
        /* reverse step 2: the node pair's block travels back */
        memcpy(gS, gR, (size_t)(L.nu * s));
        /* reverse steps 1 and 0: per source element, groups by destination node */
        int64_t n = 0;
        for (int64_t q = 0; q < L.nu; q++) {
            t1[n].row = L.u[q].rep_src_off;
            t1[n].group = L.u[q].b;
            t1[n].o1 = q;
            t1[n].o2 = 0;
            t1[n].val = gS + q * s;
            n++;
        }
        for (int r = 0; r < pt->P; r++)
            for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
                int d = pt->dests[e];
                if (node_of(pt, r) != node_of(pt, d)) continue;
                int64_t i = L.match[e];
                for (int64_t k = 0; k < pt->sendcounts[e]; k++) {
                    int64_t p = pt->rdispls[i] + k;
                    t1[n].row = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                    t1[n].group = node_of(pt, d);
                    t1[n].o1 = d;
                    t1[n].o2 = p;
                    t1[n].val = grad_recv + pt->recv_base[d] + p * s;
                    n++;
                }
            }
        qsort(t1, n, sizeof(term_t), cmp_term);
        fold_rows(t1, n, dtype, s, accumulate, grad_send, gacc, racc);
        free(gR); free(gS); free(t3); free(t1);
        loc_free(&L);
    } else {
        err = ORC_ERR_ARG;
    }
    free(gacc);
    free(racc);
    return err;
}

/* ---------------------------------------------- neighbourhood all-to-all-w --- */

/* MPI_Neighbor_alltoallw (the neighbourhood collectives of section 2.2 with one datatype
 * per edge), with the MPI standard's meaning.  A datatype here is a block of `blocklen`
 * bytes repeated over up to three strided levels (innermost first: count[0] blocks
 * stride[0] bytes apart, count[1] such rows stride[1] apart, count[2] planes stride[2]
 * apart), and `count` items of the type lie `extent` bytes apart: an hvector nested up to
 * three times and resized to `extent`, lower bound 0.  The message of an edge is the
 * sequence of bytes in type-map order (item, then level 2, level 1, level 0, then byte
 * within the block); out-edge e of r to d sends sendcounts[e] items of its send type from
 * byte sdispls[e] of r's region, in-edge i of d receives recvcounts[i] items of its
 * receive type at byte rdispls[i] of d's region, and the two byte sequences must have the
 * same length.  Errors, the smallest code winning: a bad type or type index -> ARG;
 * unmatched edge or unequal lengths or a negative count -> TRUNCATE; a negative base or
 * displacement, or a byte outside its buffer -> INDEX; a receive byte written twice ->
 * OVERLAP. */
typedef struct { int64_t blocklen, count[3], stride[3], extent; } orc_type;

typedef struct {
    int P;
    const int *in_ptr, *sources, *out_ptr, *dests;
    const int *sendcounts, *sendtypes;  /* one per out-edge */
    const int64_t *sdispls;             /* bytes            */
    const int *recvcounts, *recvtypes;  /* one per in-edge  */
    const int64_t *rdispls;             /* bytes            */
    const int64_t *send_base, *recv_base;
    const orc_type *types;
    int ntypes;
    int64_t sendbuf_bytes, recvbuf_bytes;
} orc_wpattern;

#define ORC_TYPE_MAX_SIZE ((int64_t)1 << 31)

static int64_t type_size(const orc_type *t) {
    return t->blocklen * t->count[0] * t->count[1] * t->count[2];
}

static int type_valid(const orc_type *t) {
    if (t->blocklen < 0 || t->extent < 0) return 0;
    int64_t size = t->blocklen;
    for (int l = 0; l < 3; l++) {
        if (t->count[l] < 0 || t->stride[l] < 0) return 0;
        if (t->count[l] > 0 && size > ORC_TYPE_MAX_SIZE / t->count[l]) return 0;
        size *= t->count[l];
    }
    return size <= ORC_TYPE_MAX_SIZE;
}

/* Byte offset (from the message's displacement) of byte b of the message. */
static int64_t type_byte(const orc_type *t, int64_t b) {
    int64_t size = type_size(t);
    int64_t item = b / size, w = b % size;
    int64_t blk = w / t->blocklen, off = w % t->blocklen;
    int64_t c0 = blk % t->count[0];
    blk /= t->count[0];
    int64_t c1 = blk % t->count[1];
    int64_t c2 = blk / t->count[1];
    return item * t->extent + c2 * t->stride[2] + c1 * t->stride[1] + c0 * t->stride[0] + off;
}

/* Matches the edges and checks everything; returns the smallest error code found. */
static int w_prepare(const orc_wpattern *wp, int64_t **match_out) {
    if (!wp || wp->P <= 0 || !wp->in_ptr || !wp->out_ptr || wp->ntypes < 0 || (wp->ntypes && !wp->types))
        return ORC_ERR_ARG;
    for (int k = 0; k < wp->ntypes; k++)
        if (!type_valid(&wp->types[k])) return ORC_ERR_ARG;
    orc_pattern g;
    memset(&g, 0, sizeof(g));
    g.P = wp->P;
    g.ppn = 1;
    g.in_ptr = wp->in_ptr; g.sources = wp->sources; g.out_ptr = wp->out_ptr; g.dests = wp->dests;
    int64_t n_out = wp->out_ptr[wp->P] > 0 ? wp->out_ptr[wp->P] : 1;
    int64_t *match = malloc(sizeof(int64_t) * n_out);
    if (!match) return ORC_ERR_NOMEM;
    int err = orc_match(&g, match);
    if (err) { free(match); return err; }
    if (wp->out_ptr[wp->P] > 0 && (!wp->sendcounts || !wp->sendtypes || !wp->sdispls || !wp->recvcounts ||
                                   !wp->recvtypes || !wp->rdispls))
        err = ORC_ERR_ARG;
    if (!wp->send_base || !wp->recv_base) err = ORC_ERR_ARG;
    if (err) { free(match); return err; }
    for (int r = 0; r < wp->P; r++)
        if (wp->send_base[r] < 0 || wp->recv_base[r] < 0) MIN_ERR(err, ORC_ERR_INDEX);
    for (int r = 0; r < wp->P; r++)
        for (int64_t e = wp->out_ptr[r]; e < wp->out_ptr[r + 1]; e++) {
            int d = wp->dests[e];
            int64_t i = match[e];
            int ts = wp->sendtypes[e], tr = wp->recvtypes[i];
            if (ts < 0 || ts >= wp->ntypes || tr < 0 || tr >= wp->ntypes) { MIN_ERR(err, ORC_ERR_ARG); continue; }
            const orc_type *Ts = &wp->types[ts], *Tr = &wp->types[tr];
            int64_t n = (int64_t)wp->sendcounts[e] * type_size(Ts);
            if (wp->sendcounts[e] < 0 || wp->recvcounts[i] < 0 || n != (int64_t)wp->recvcounts[i] * type_size(Tr)) {
                MIN_ERR(err, ORC_ERR_TRUNCATE);
                continue;
            }
            if (wp->sdispls[e] < 0 || wp->rdispls[i] < 0) { MIN_ERR(err, ORC_ERR_INDEX); continue; }
            if (wp->send_base[r] < 0 || wp->recv_base[d] < 0) continue;
            for (int64_t b = 0; b < n; b++) {
                int64_t sa = wp->send_base[r] + wp->sdispls[e] + type_byte(Ts, b);
                int64_t da = wp->recv_base[d] + wp->rdispls[i] + type_byte(Tr, b);
                if (sa >= wp->sendbuf_bytes || da >= wp->recvbuf_bytes) { MIN_ERR(err, ORC_ERR_INDEX); break; }
            }
        }
    if (err == ORC_OK && wp->recvbuf_bytes > 0) {
        uint8_t *seen = calloc((size_t)wp->recvbuf_bytes, 1);
        if (!seen) { free(match); return ORC_ERR_NOMEM; }
        for (int r = 0; r < wp->P && !err; r++)
            for (int64_t e = wp->out_ptr[r]; e < wp->out_ptr[r + 1] && !err; e++) {
                int d = wp->dests[e];
                int64_t i = match[e];
                const orc_type *Tr = &wp->types[wp->recvtypes[i]];
                int64_t n = (int64_t)wp->recvcounts[i] * type_size(Tr);
                for (int64_t b = 0; b < n; b++) {
                    int64_t da = wp->recv_base[d] + wp->rdispls[i] + type_byte(Tr, b);
                    if (seen[da]) { err = ORC_ERR_OVERLAP; break; }
                    seen[da] = 1;
                }
            }
        free(seen);
    }
    if (err) { free(match); return err; }
    *match_out = match;
    return ORC_OK;
}

int orc_alltoallw_validate(const orc_wpattern *wp) {
    int64_t *match = NULL;
    int err = w_prepare(wp, &match);
    free(match);
    return err;
}

/* The definition: every byte b of every message is copied from its send address to its
 * receive address; receive bytes no message covers are untouched. */
int orc_alltoallw(const orc_wpattern *wp, const uint8_t *sendbuf, uint8_t *recvbuf) {
    int64_t *match = NULL;
    int err = w_prepare(wp, &match);
    if (err) return err;
    for (int r = 0; r < wp->P; r++)
        for (int64_t e = wp->out_ptr[r]; e < wp->out_ptr[r + 1]; e++) {
            int d = wp->dests[e];
            int64_t i = match[e];
            const orc_type *Ts = &wp->types[wp->sendtypes[e]], *Tr = &wp->types[wp->recvtypes[i]];
            int64_t n = (int64_t)wp->sendcounts[e] * type_size(Ts);
            for (int64_t b = 0; b < n; b++)
                recvbuf[wp->recv_base[d] + wp->rdispls[i] + type_byte(Tr, b)] =
                    sendbuf[wp->send_base[r] + wp->sdispls[e] + type_byte(Ts, b)];
        }
    free(match);
    return ORC_OK;
}

/* Reverse exchange of the all-to-all-w in the standard order: every payload element
 * (4 or 8 bytes, aligned with the message byte sequence) of the send buffer receives the
 * left-to-right sum of the gradients at the receive addresses it was copied to, ordered
 * by (destination rank, receive address); accumulate adds the sum to the old value;
 * elements no message reads are untouched.  Every block length, stride, extent, base and
 * displacement must be a multiple of the payload size (else ARG), so that each payload
 * element travels whole. */
int orc_alltoallw_backward(const orc_wpattern *wp, int dtype, int accumulate, const uint8_t *grad_recv,
                           uint8_t *grad_send) {
    if (dtype != ORC_F32 && dtype != ORC_F64) return ORC_ERR_ARG;
    int64_t dsz = dtype == ORC_F64 ? 8 : 4;
    int64_t *match = NULL;
    int err = w_prepare(wp, &match);
    if (err) return err;
    for (int k = 0; k < wp->ntypes; k++) {
        const orc_type *t = &wp->types[k];
        if (type_size(t) == 0) continue;
        if (t->blocklen % dsz || t->stride[0] % dsz || t->stride[1] % dsz || t->stride[2] % dsz || t->extent % dsz)
            err = ORC_ERR_ARG;
    }
    int64_t n_terms = 0;
    for (int r = 0; r < wp->P && !err; r++) {
        if (wp->send_base[r] % dsz || wp->recv_base[r] % dsz) err = ORC_ERR_ARG;
        for (int64_t e = wp->out_ptr[r]; e < wp->out_ptr[r + 1]; e++) {
            int64_t i = match[e];
            if (wp->sdispls[e] % dsz || wp->rdispls[i] % dsz) err = ORC_ERR_ARG;
            n_terms += (int64_t)wp->sendcounts[e] * type_size(&wp->types[wp->sendtypes[e]]) / dsz;
        }
    }
    if (err) { free(match); return err; }
    term_t *t = malloc(sizeof(term_t) * (n_terms ? n_terms : 1));
    uint8_t *gacc = malloc((size_t)dsz), *racc = malloc((size_t)dsz);
    if (!t || !gacc || !racc) { free(t); free(gacc); free(racc); free(match); return ORC_ERR_NOMEM; }
    int64_t n = 0;
    for (int r = 0; r < wp->P; r++)
        for (int64_t e = wp->out_ptr[r]; e < wp->out_ptr[r + 1]; e++) {
            int d = wp->dests[e];
            int64_t i = match[e];
            const orc_type *Ts = &wp->types[wp->sendtypes[e]], *Tr = &wp->types[wp->recvtypes[i]];
            int64_t len = (int64_t)wp->sendcounts[e] * type_size(Ts);
            for (int64_t b = 0; b < len; b += dsz) {
                int64_t da = wp->recv_base[d] + wp->rdispls[i] + type_byte(Tr, b);
                t[n].row = wp->send_base[r] + wp->sdispls[e] + type_byte(Ts, b);
                t[n].group = 0;
                t[n].o1 = d;
                t[n].o2 = da;
                t[n].val = grad_recv + da;
                n++;
            }
        }
    qsort(t, n, sizeof(term_t), cmp_term);
    fold_rows(t, n, dtype, dsz, accumulate, grad_send, gacc, racc);
    free(t);
    free(gacc);
    free(racc);
    free(match);
    return ORC_OK;
}

/* ------------------------------------------------------ partitioned exchange --- */

/* Partitioned communication (section 2.3): a persistent exchange whose send buffer is cut
 * into partitions that the producer marks ready one by one; each ready partition's data
 * may move before the rest of the buffer exists ("early-bird"), and a receive partition
 * is complete once every value landing in it has arrived.  Partition p of the send buffer
 * is the byte range [part_ptr[p], part_ptr[p+1]); the pointers start at 0, never decrease
 * and end at the buffer's size, and no element may straddle a boundary (else ARG).  The
 * same holds for receive partitions over the receive buffer. */
static int check_parts(int n, const int64_t *ptr, int64_t bytes) {
    if (n < 1 || !ptr || ptr[0] != 0 || ptr[n] != bytes) return ORC_ERR_ARG;
    for (int p = 0; p < n; p++)
        if (ptr[p + 1] < ptr[p]) return ORC_ERR_ARG;
    return ORC_OK;
}

/* The partition holding bytes [off, off + s), or -1 when they straddle a boundary. */
static int part_of(int n, const int64_t *ptr, int64_t off, int64_t s) {
    for (int p = 0; p < n; p++)
        if (ptr[p] <= off && off < ptr[p + 1]) return off + s <= ptr[p + 1] ? p : -1;
    return -1;
}

/* Every element's (send partition, receive partition); -1 entries make the call fail. */
static int part_scan(const orc_pattern *pt, const int64_t *match, int npart, const int64_t *part_ptr, int nrpart,
                     const int64_t *rpart_ptr, int *sp, int *rp) {
    int64_t s = pt->elem_size, n = 0;
    for (int r = 0; r < pt->P; r++)
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            int64_t i = match[e];
            for (int64_t k = 0; k < pt->sendcounts[e]; k++, n++) {
                int64_t src = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                int64_t dst = pt->recv_base[d] + (pt->rdispls[i] + k) * s;
                sp[n] = part_of(npart, part_ptr, src, s);
                rp[n] = rpart_ptr ? part_of(nrpart, rpart_ptr, dst, s) : 0;
                if (sp[n] < 0 || rp[n] < 0) return ORC_ERR_ARG;
            }
        }
    return ORC_OK;
}

/* The exchange after the partitions with ready[p] != 0 have moved: a receive element is
 * written when its source element lies in a ready partition, else left as it was. */
int orc_standard_partial(const orc_pattern *pt, int npart, const int64_t *part_ptr, const uint8_t *ready,
                         const uint8_t *sendbuf, uint8_t *recvbuf) {
    int64_t *match = NULL;
    int err = prepare(pt, &match);
    if (err) return err;
    if (check_parts(npart, part_ptr, pt->sendbuf_bytes)) { free(match); return ORC_ERR_ARG; }
    int64_t V = 0;
    for (int64_t e = 0; e < pt->out_ptr[pt->P]; e++) V += pt->sendcounts[e];
    int *sp = malloc(sizeof(int) * (V ? V : 1)), *rp = malloc(sizeof(int) * (V ? V : 1));
    if (!sp || !rp) { free(sp); free(rp); free(match); return ORC_ERR_NOMEM; }
    err = part_scan(pt, match, npart, part_ptr, 0, NULL, sp, rp);
    int64_t s = pt->elem_size, n = 0;
    for (int r = 0; r < pt->P && !err; r++)
        for (int64_t e = pt->out_ptr[r]; e < pt->out_ptr[r + 1]; e++) {
            int d = pt->dests[e];
            int64_t i = match[e];
            for (int64_t k = 0; k < pt->sendcounts[e]; k++, n++) {
                if (!ready[sp[n]]) continue;
                int64_t src = pt->send_base[r] + send_elem(pt, r, pt->sdispls[e] + k) * s;
                int64_t dst = pt->recv_base[d] + (pt->rdispls[i] + k) * s;
                memcpy(recvbuf + dst, sendbuf + src, (size_t)s);
            }
        }
    free(sp); free(rp); free(match);
    return err;
}

/* arrived[j] = 1 when every element received into receive partition j comes from a ready
 * send partition (a partition that receives nothing has arrived). */
int orc_arrived(const orc_pattern *pt, int npart, const int64_t *part_ptr, const uint8_t *ready, int nrpart,
                const int64_t *rpart_ptr, uint8_t *arrived) {
    int64_t *match = NULL;
    int err = prepare(pt, &match);
    if (err) return err;
    if (check_parts(npart, part_ptr, pt->sendbuf_bytes) || check_parts(nrpart, rpart_ptr, pt->recvbuf_bytes)) {
        free(match);
        return ORC_ERR_ARG;
    }
    int64_t V = 0;
    for (int64_t e = 0; e < pt->out_ptr[pt->P]; e++) V += pt->sendcounts[e];
    int *sp = malloc(sizeof(int) * (V ? V : 1)), *rp = malloc(sizeof(int) * (V ? V : 1));
    if (!sp || !rp) { free(sp); free(rp); free(match); return ORC_ERR_NOMEM; }
    err = part_scan(pt, match, npart, part_ptr, nrpart, rpart_ptr, sp, rp);
    if (!err) {
        for (int j = 0; j < nrpart; j++) arrived[j] = 1;
        for (int64_t n = 0; n < V; n++)
            if (!ready[sp[n]]) arrived[rp[n]] = 0;
    }
    free(sp); free(rp); free(match);
    return err;
}

/* -------------------------------------------- derived neighbourhood collectives --- */

/* MPI Advance offers its persistent neighbourhood collectives as drop-in replacements of
 * the MPI calls (section 2.2) and its all-to-all-v over the whole communicator as
 * MPIX_Alltoallv (section 2.1, Listing 2).  Their meaning is the MPI standard's, and each
 * is a neighbourhood all-to-all-v with counts and displacements fixed by the call:
 *   mode 0, MPI_Neighbor_alltoall(count): rank r sends `count` elements starting at
 *     element j*count of its send region to its j-th out-neighbour; rank d stores the
 *     `count` elements coming from its i-th in-neighbour at element i*count of its
 *     receive region;
 *   mode 1, MPI_Neighbor_allgather(count): rank r sends the same elements [0, count) of
 *     its send region to every out-neighbour; rank d stores the block from its i-th
 *     in-neighbour at element i*count;
 *   mode 2, MPI_Neighbor_allgatherv(sendcount[r], recvcounts, rdispls): rank r sends its
 *     elements [0, sendcount[r]) to every out-neighbour; rank d receives recvcounts[i]
 *     elements from its i-th in-neighbour at element rdispls[i] (given by the caller, so
 *     only the send side is derived here).
 * "j-th" and "i-th" are positions in the rank's own out- and in-list.  A repeated
 * neighbour is paired by the multigraph rule of orc_match, like every other exchange.
 * This fills the per-out-edge sendcounts / sdispls and, for modes 0 and 1, the per-in-edge
 * recvcounts / rdispls.  Errors: the graph's own (orc_match), ORC_ERR_ARG for a negative
 * count or a missing array, ORC_ERR_UNSUPPORTED when a derived displacement exceeds the
 * int32 range of the all-to-all-v arguments. */
int orc_derive_neighbor(const orc_pattern *g, int mode, int count, const int *rank_count, int *sendcounts,
                        int *sdispls, int *recvcounts, int *rdispls) {
    if (!g || g->P <= 0 || !g->in_ptr || !g->out_ptr || mode < 0 || mode > 2) return ORC_ERR_ARG;
    int P = g->P;
    int64_t n = g->out_ptr[P] > 0 ? g->out_ptr[P] : 1;
    int64_t *match = malloc(sizeof(int64_t) * n);
    if (!match) return ORC_ERR_NOMEM;
    int err = orc_match(g, match);
    free(match);
    if (err) return err;
    if ((mode != 2 && count < 0) || (mode == 2 && !rank_count)) return ORC_ERR_ARG;
    if (!sendcounts || !sdispls || (mode != 2 && (!recvcounts || !rdispls))) return ORC_ERR_ARG;
    for (int r = 0; r < P; r++)
        for (int64_t e = g->out_ptr[r]; e < g->out_ptr[r + 1]; e++) {
            int64_t j = e - g->out_ptr[r];     /* position of this neighbour in r's out-list */
            int64_t disp = mode == 0 ? j * (int64_t)count : 0;
            if (disp > INT32_MAX) err = ORC_ERR_UNSUPPORTED;
            sendcounts[e] = mode == 2 ? rank_count[r] : count;
            sdispls[e] = disp > INT32_MAX ? 0 : (int)disp;
        }
    if (mode != 2)
        for (int d = 0; d < P; d++)
            for (int64_t i = g->in_ptr[d]; i < g->in_ptr[d + 1]; i++) {
                int64_t k = i - g->in_ptr[d];  /* position of this neighbour in d's in-list */
                int64_t disp = k * (int64_t)count;
                if (disp > INT32_MAX) err = ORC_ERR_UNSUPPORTED;
                recvcounts[i] = count;
                rdispls[i] = disp > INT32_MAX ? 0 : (int)disp;
            }
    return err;
}

/* The communicator of MPIX_Alltoallv as a distributed graph: every rank lists every rank,
 * itself included, in rank order, in both its in- and out-list.  Rank r's out-edge to d is
 * then edge r*P + d and d's in-edge from r is edge d*P + r, so the P x P count and
 * displacement matrices of the call (row-major by rank) are the per-edge arrays as they
 * are.  ptr has P+1 entries, ranks P*P; ORC_ERR_UNSUPPORTED when P*P exceeds int32. */
int orc_complete_graph(int P, int *ptr, int *ranks) {
    if (P <= 0 || !ptr || !ranks) return ORC_ERR_ARG;
    if ((int64_t)P * P > INT32_MAX) return ORC_ERR_UNSUPPORTED;
    for (int r = 0; r <= P; r++) ptr[r] = r * P;
    for (int r = 0; r < P; r++)
        for (int d = 0; d < P; d++) ranks[(int64_t)r * P + d] = d;
    return ORC_OK;
}
