/*
 * mg_oracle.c -- CPU oracle for the Mixture Graph hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Arithmetic: exact integers (uint64) for mixtures, node keys and histograms;
 * IEEE fp64 for colours.  Every function cites the passage of the paper it
 * follows:
 *   Eq. 4 (Sec. 3.1)       normalised histogram mipmap
 *   Eq. 5-8 (Sec. 3.2)     factorisation into binary lerps, the DAG
 *   Sec. 3.3               re-use (pruning) of identical nodes
 *   Sec. 3.4, Fig. 5       topological level of every node
 *   Sec. 3.4, Sec. 4       colour propagation, paletted lookup
 *   Sec. 3.6, Algorithm 1  footprint assembly of a box query
 *   Sec. 4                 ray marching through the node values (LOD,
 *                          interpolation, opacity correction, empty-space
 *                          skipping)
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   R1 border normalisation: N counts children in support (Eq. 4), so a level
 *      l mixture is stored as integers c = 8^l * H, with c_parent =
 *      (8/N) * sum(c_child), exact because N is 1, 2, 4 or 8.
 *   R2 sources are the segment IDs 0..S-1 (0-based).
 *   R3 pair choice: the balanced positional pairing.  The entries of a mixture
 *      are sorted by segment ID; each round lerps positions (0,1),(2,3),...
 *      and carries an odd last entry to the end of the next round's list,
 *      until one entry remains.  (The paper lets any pair be picked.)
 *   R4 a node is the key (p, q, a, b): the lerp (a*p + b*q)/(a+b) of its two
 *      predecessors with coprime integer weights a, b >= 1.  Identical keys are
 *      one node (exact ratios, no quantiser).
 *   R5 canonical node IDs: sources keep their segment ID; internal nodes are
 *      numbered S, S+1, ... in ascending (depth, p', q', a, b), where p', q'
 *      are the canonical IDs of the predecessors.
 *   R6 Algorithm 1: "lzcnt(x)" is floor(log2 x); tzcnt(0) is infinite; the
 *      sample position advances by the block size after each block.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MGO_MAX_LEVELS 40
#define MGO_NONE 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Eq. 4 (Sec. 3.1): resolution of every level, rounding up at each level    */
/* until the level with 1^3 voxels.                                          */
/* ------------------------------------------------------------------------ */
int mgo_level_dims(int64_t nx, int64_t ny, int64_t nz, int64_t *dims_out, int max_levels)
{
    int64_t d[3] = {nx, ny, nz};
    int L = 0;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    for (;;) {
        if (L >= max_levels) return -1;
        dims_out[3 * L + 0] = d[0];
        dims_out[3 * L + 1] = d[1];
        dims_out[3 * L + 2] = d[2];
        L++;
        if (d[0] == 1 && d[1] == 1 && d[2] == 1) break;
        for (int k = 0; k < 3; k++) d[k] = (d[k] + 1) / 2;
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Mixture lists of one level: per voxel a list of (segment id, count),      */
/* sorted by id, with count = 8^l * H (reading R1).                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t d[3];
    int64_t nv;       /* voxels */
    int64_t nnz;      /* entries */
    uint64_t *off;    /* nv + 1 */
    uint32_t *ids;    /* nnz */
    uint64_t *cnt;    /* nnz */
} mgo_lists;

static void lists_free(mgo_lists *m)
{
    free(m->off); free(m->ids); free(m->cnt);
    memset(m, 0, sizeof(*m));
}

static uint32_t vol_id(const void *vol, int id_bytes, int64_t i)
{
    if (id_bytes == 2) return ((const uint16_t *)vol)[i];
    return ((const uint32_t *)vol)[i];
}

/* Level 0: H(v,0) is the unit vector of the voxel's segment ID (Eq. 4). */
static int lists_level0(const void *vol, int id_bytes, int64_t nx, int64_t ny, int64_t nz, mgo_lists *m)
{
    m->d[0] = nx; m->d[1] = ny; m->d[2] = nz;
    m->nv = nx * ny * nz;
    m->nnz = m->nv;
    m->off = (uint64_t *)malloc((size_t)(m->nv + 1) * sizeof(uint64_t));
    m->ids = (uint32_t *)malloc((size_t)m->nv * sizeof(uint32_t));
    m->cnt = (uint64_t *)malloc((size_t)m->nv * sizeof(uint64_t));
    if (!m->off || !m->ids || !m->cnt) return -1;
    for (int64_t i = 0; i < m->nv; i++) {
        m->off[i] = (uint64_t)i;
        m->ids[i] = vol_id(vol, id_bytes, i);
        m->cnt[i] = 1;
    }
    m->off[m->nv] = (uint64_t)m->nv;
    return 0;
}

typedef struct { uint32_t id; uint64_t c; } pair_ic;

static int cmp_pair_ic(const void *x, const void *y)
{
    const pair_ic *a = (const pair_ic *)x, *b = (const pair_ic *)y;
    return (a->id > b->id) - (a->id < b->id);
}

/* Eq. 4: the parent mixture is the average of the children in its support,
 * N of them.  In the integer form (R1): c_parent = (8/N) * sum of children. */
static int lists_next(const mgo_lists *in, mgo_lists *out)
{
    int64_t dn[3];
    for (int k = 0; k < 3; k++) dn[k] = (in->d[k] + 1) / 2;
    out->d[0] = dn[0]; out->d[1] = dn[1]; out->d[2] = dn[2];
    out->nv = dn[0] * dn[1] * dn[2];
    /* entries never grow from one level to the next */
    out->off = (uint64_t *)malloc((size_t)(out->nv + 1) * sizeof(uint64_t));
    out->ids = (uint32_t *)malloc((size_t)(in->nnz > 0 ? in->nnz : 1) * sizeof(uint32_t));
    out->cnt = (uint64_t *)malloc((size_t)(in->nnz > 0 ? in->nnz : 1) * sizeof(uint64_t));
    if (!out->off || !out->ids || !out->cnt) return -1;
    size_t cap = 64;
    pair_ic *tmp = (pair_ic *)malloc(cap * sizeof(pair_ic));
    if (!tmp) return -1;
    int64_t w = 0;
    for (int64_t Z = 0; Z < dn[2]; Z++)
    for (int64_t Y = 0; Y < dn[1]; Y++)
    for (int64_t X = 0; X < dn[0]; X++) {
        int64_t v = (Z * dn[1] + Y) * dn[0] + X;
        out->off[v] = (uint64_t)w;
        size_t n = 0;
        int N = 0;
        for (int k = 0; k < 2; k++)
        for (int j = 0; j < 2; j++)
        for (int i = 0; i < 2; i++) {
            int64_t x = 2 * X + i, y = 2 * Y + j, z = 2 * Z + k;
            if (x >= in->d[0] || y >= in->d[1] || z >= in->d[2]) continue;
            N++;
            int64_t c = (z * in->d[1] + y) * in->d[0] + x;
            for (uint64_t e = in->off[c]; e < in->off[c + 1]; e++) {
                if (n == cap) {
                    cap *= 2;
                    pair_ic *t2 = (pair_ic *)realloc(tmp, cap * sizeof(pair_ic));
                    if (!t2) { free(tmp); return -1; }
                    tmp = t2;
                }
                tmp[n].id = in->ids[e];
                tmp[n].c = in->cnt[e];
                n++;
            }
        }
        qsort(tmp, n, sizeof(pair_ic), cmp_pair_ic);
        uint64_t scale = (uint64_t)(8 / N);
        for (size_t e = 0; e < n;) {
            uint32_t id = tmp[e].id;
            uint64_t s = 0;
            while (e < n && tmp[e].id == id) { s += tmp[e].c; e++; }
            out->ids[w] = id;
            out->cnt[w] = s * scale;
            w++;
        }
    }
    out->off[out->nv] = (uint64_t)w;
    out->nnz = w;
    free(tmp);
    return 0;
}

/* Mixture lists of one level of the volume, for tests: returns a heap block
 * the caller copies out and frees with mgo_level_release. */
typedef struct {
    int64_t nv, nnz;
    uint64_t *off;
    uint32_t *ids;
    uint64_t *cnt;
} mgo_level_out;

int mgo_mixtures(const void *vol, int id_bytes, int64_t nx, int64_t ny, int64_t nz,
                 int level, mgo_level_out *out)
{
    mgo_lists cur, nxt;
    memset(&cur, 0, sizeof(cur));
    if (lists_level0(vol, id_bytes, nx, ny, nz, &cur)) return -1;
    for (int l = 0; l < level; l++) {
        memset(&nxt, 0, sizeof(nxt));
        if (lists_next(&cur, &nxt)) { lists_free(&cur); return -1; }
        lists_free(&cur);
        cur = nxt;
    }
    out->nv = cur.nv; out->nnz = cur.nnz;
    out->off = cur.off; out->ids = cur.ids; out->cnt = cur.cnt;
    return 0;
}

void mgo_level_release(mgo_level_out *out)
{
    free(out->off); free(out->ids); free(out->cnt);
    memset(out, 0, sizeof(*out));
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2-3.3: factorisation into binary lerps with re-use of identical     */
/* nodes.  Plain open-addressing map from key (p, q, a, b) to a temporary     */
/* node number in order of creation.                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* node arrays, indexed by temporary number; sources are 0..S-1 */
    uint32_t *p, *q;
    uint64_t *a, *b;
    int32_t *depth;
    int64_t n, cap;
    /* map */
    int64_t *slot;    /* -1 = empty, else node number */
    int64_t nslot;    /* power of two */
} mgo_table;

static uint64_t mix64(uint64_t x)
{
    x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

static uint64_t key_hash(uint32_t p, uint32_t q, uint64_t a, uint64_t b)
{
    uint64_t h = mix64(((uint64_t)p << 32) | q);
    h = mix64(h ^ a);
    h = mix64(h ^ (b * 0x9e3779b97f4a7c15ULL));
    return h;
}

static int table_grow_nodes(mgo_table *t)
{
    int64_t nc = t->cap ? t->cap * 2 : 1024;
    uint32_t *np_ = (uint32_t *)realloc(t->p, (size_t)nc * sizeof(uint32_t));
    if (!np_) return -1;
    t->p = np_;
    uint32_t *nq = (uint32_t *)realloc(t->q, (size_t)nc * sizeof(uint32_t));
    if (!nq) return -1;
    t->q = nq;
    uint64_t *na = (uint64_t *)realloc(t->a, (size_t)nc * sizeof(uint64_t));
    if (!na) return -1;
    t->a = na;
    uint64_t *nb = (uint64_t *)realloc(t->b, (size_t)nc * sizeof(uint64_t));
    if (!nb) return -1;
    t->b = nb;
    int32_t *nd = (int32_t *)realloc(t->depth, (size_t)nc * sizeof(int32_t));
    if (!nd) return -1;
    t->depth = nd;
    t->cap = nc;
    return 0;
}

static int table_rehash(mgo_table *t, int64_t nslot)
{
    int64_t *s = (int64_t *)malloc((size_t)nslot * sizeof(int64_t));
    if (!s) return -1;
    for (int64_t i = 0; i < nslot; i++) s[i] = -1;
    free(t->slot);
    t->slot = s;
    t->nslot = nslot;
    return 0;
}

static int table_init(mgo_table *t, uint32_t S)
{
    memset(t, 0, sizeof(*t));
    while (t->cap < (int64_t)S + 1) if (table_grow_nodes(t)) return -1;
    for (uint32_t s = 0; s < S; s++) {
        t->p[s] = MGO_NONE; t->q[s] = MGO_NONE; t->a[s] = 0; t->b[s] = 0; t->depth[s] = 0;
    }
    t->n = S;
    return table_rehash(t, 1024);
}

static void table_free(mgo_table *t)
{
    free(t->p); free(t->q); free(t->a); free(t->b); free(t->depth); free(t->slot);
    memset(t, 0, sizeof(*t));
}

static void table_insert_slot(mgo_table *t, int64_t node)
{
    uint64_t h = key_hash(t->p[node], t->q[node], t->a[node], t->b[node]);
    int64_t m = t->nslot - 1;
    int64_t i = (int64_t)(h & (uint64_t)m);
    while (t->slot[i] >= 0) i = (i + 1) & m;
    t->slot[i] = node;
}

static uint64_t gcd_u64(uint64_t x, uint64_t y)
{
    while (y) { uint64_t r = x % y; x = y; y = r; }
    return x;
}

/* The node with key (p, q, a, b), created if new (Sec. 3.3 re-use). */
static int64_t table_get_key(mgo_table *t, uint32_t p, uint32_t q, uint64_t a, uint64_t b)
{
    uint64_t h = key_hash(p, q, a, b);
    int64_t m = t->nslot - 1;
    int64_t i = (int64_t)(h & (uint64_t)m);
    while (t->slot[i] >= 0) {
        int64_t k = t->slot[i];
        if (t->p[k] == p && t->q[k] == q && t->a[k] == a && t->b[k] == b) return k;
        i = (i + 1) & m;
    }
    if (t->n == t->cap) if (table_grow_nodes(t)) return -1;
    int64_t k = t->n++;
    t->p[k] = p; t->q[k] = q; t->a[k] = a; t->b[k] = b;
    /* Sec. 3.4: topological level = max(level of predecessors) + 1 */
    int32_t dp = t->depth[p], dq = t->depth[q];
    t->depth[k] = (dp > dq ? dp : dq) + 1;
    t->slot[i] = k;
    if (2 * (t->n) > t->nslot) {
        if (table_rehash(t, t->nslot * 2)) return -1;
        for (int64_t j = 0; j < t->n; j++) if (t->p[j] != MGO_NONE) table_insert_slot(t, j);
    }
    return k;
}

/* Eq. 5-6: the lerp of the entries (p, wp) and (q, wq) with the reduced ratio
 * a:b = wp:wq; an identical key already in the table is re-used (Sec. 3.3). */
static int64_t table_get(mgo_table *t, uint32_t p, uint64_t wp, uint32_t q, uint64_t wq)
{
    uint64_t g = gcd_u64(wp, wq);
    return table_get_key(t, p, q, wp / g, wq / g);
}

/* Reading R3: factorise one mixture (entries sorted by id) with the balanced
 * positional pairing; returns the node representing the whole mixture. */
static int64_t factor_one(mgo_table *t, const uint32_t *ids, const uint64_t *cnt, int64_t n,
                          uint32_t *node_buf, uint64_t *w_buf)
{
    for (int64_t k = 0; k < n; k++) { node_buf[k] = ids[k]; w_buf[k] = cnt[k]; }
    while (n > 1) {
        int64_t m = 0;
        for (int64_t k = 0; k + 1 < n; k += 2) {
            int64_t nd = table_get(t, node_buf[k], w_buf[k], node_buf[k + 1], w_buf[k + 1]);
            if (nd < 0) return -1;
            uint64_t w = w_buf[k] + w_buf[k + 1];
            node_buf[m] = (uint32_t)nd;
            w_buf[m] = w;
            m++;
        }
        if (n & 1) { node_buf[m] = node_buf[n - 1]; w_buf[m] = w_buf[n - 1]; m++; }
        n = m;
    }
    return node_buf[0];
}

/* ------------------------------------------------------------------------ */
/* The whole graph (Sec. 3.2-3.4).                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t S;
    int L;
    int64_t dims[MGO_MAX_LEVELS * 3];
    int64_t N;          /* nodes including sources */
    int D;              /* topological depth */
    uint32_t *p, *q;    /* canonical order */
    uint64_t *a, *b;
    int32_t *depth;
    int64_t *bucket;    /* D + 2 offsets: bucket d = [bucket[d], bucket[d+1]) */
    uint32_t **mip;     /* per level, canonical node ID of every voxel */
    int64_t max_nnz;    /* longest mixture list of any voxel */
    int64_t pairs;      /* sum over voxels of (nnz - 1) */
    int64_t *canon;     /* build-time only: temporary number -> canonical ID */
} mgo_graph;

typedef struct {
    uint32_t cp, cq;
    uint64_t a, b;
    int64_t tmp;
} relabel_key;

static int cmp_relabel(const void *x, const void *y)
{
    const relabel_key *u = (const relabel_key *)x, *v = (const relabel_key *)y;
    if (u->cp != v->cp) return u->cp < v->cp ? -1 : 1;
    if (u->cq != v->cq) return u->cq < v->cq ? -1 : 1;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    if (u->b != v->b) return u->b < v->b ? -1 : 1;
    return 0;
}

/* Reading R5: canonical numbering, depth by depth.  Fills the node arrays,
 * bucket offsets and g->canon (temporary number -> canonical ID). */
static int relabel(mgo_graph *g, mgo_table *t)
{
    uint32_t S = g->S;
    int D = 0;
    for (int64_t k = S; k < t->n; k++) if (t->depth[k] > D) D = t->depth[k];
    g->D = D;
    g->N = t->n;
    size_t n1 = (size_t)(t->n > 0 ? t->n : 1);
    g->canon = (int64_t *)malloc(n1 * sizeof(int64_t));
    g->bucket = (int64_t *)malloc((size_t)(D + 2) * sizeof(int64_t));
    g->p = (uint32_t *)malloc(n1 * sizeof(uint32_t));
    g->q = (uint32_t *)malloc(n1 * sizeof(uint32_t));
    g->a = (uint64_t *)malloc(n1 * sizeof(uint64_t));
    g->b = (uint64_t *)malloc(n1 * sizeof(uint64_t));
    g->depth = (int32_t *)malloc(n1 * sizeof(int32_t));
    relabel_key *keys = (relabel_key *)malloc(n1 * sizeof(relabel_key));
    if (!g->canon || !g->bucket || !g->p || !g->q || !g->a || !g->b || !g->depth || !keys) {
        free(keys);
        return -1;
    }
    for (uint32_t s = 0; s < S; s++) {
        g->canon[s] = s;
        g->p[s] = MGO_NONE; g->q[s] = MGO_NONE; g->a[s] = 0; g->b[s] = 0; g->depth[s] = 0;
    }
    g->bucket[0] = 0;
    g->bucket[1] = S;
    int64_t next = S;
    for (int d = 1; d <= D; d++) {
        int64_t m = 0;
        for (int64_t k = S; k < t->n; k++) {
            if (t->depth[k] != d) continue;
            keys[m].cp = (uint32_t)g->canon[t->p[k]];
            keys[m].cq = (uint32_t)g->canon[t->q[k]];
            keys[m].a = t->a[k];
            keys[m].b = t->b[k];
            keys[m].tmp = k;
            m++;
        }
        qsort(keys, (size_t)m, sizeof(relabel_key), cmp_relabel);
        for (int64_t i = 0; i < m; i++) {
            int64_t c = next + i;
            g->canon[keys[i].tmp] = c;
            g->p[c] = keys[i].cp; g->q[c] = keys[i].cq;
            g->a[c] = keys[i].a; g->b[c] = keys[i].b;
            g->depth[c] = d;
        }
        next += m;
        g->bucket[d + 1] = next;
    }
    free(keys);
    return 0;
}

void mgo_graph_free(mgo_graph *g)
{
    if (!g) return;
    free(g->p); free(g->q); free(g->a); free(g->b); free(g->depth); free(g->bucket);
    free(g->canon);
    if (g->mip) for (int l = 0; l < g->L; l++) free(g->mip[l]);
    free(g->mip);
    free(g);
}

mgo_graph *mgo_build(const void *vol, int id_bytes, int64_t nx, int64_t ny, int64_t nz, uint32_t S)
{
    mgo_graph *g = (mgo_graph *)calloc(1, sizeof(mgo_graph));
    if (!g) return NULL;
    g->S = S;
    g->L = mgo_level_dims(nx, ny, nz, g->dims, MGO_MAX_LEVELS);
    if (g->L < 1) { free(g); return NULL; }
    int64_t V0 = nx * ny * nz;
    for (int64_t i = 0; i < V0; i++) if (vol_id(vol, id_bytes, i) >= S) { free(g); return NULL; }
    g->mip = (uint32_t **)calloc((size_t)g->L, sizeof(uint32_t *));
    mgo_table t;
    if (table_init(&t, S)) { mgo_graph_free(g); return NULL; }

    /* level 0: the mip ID is the segment ID (Sec. 3.4, lossless level 0) */
    g->mip[0] = (uint32_t *)malloc((size_t)V0 * sizeof(uint32_t));
    for (int64_t i = 0; i < V0; i++) g->mip[0][i] = vol_id(vol, id_bytes, i);

    mgo_lists cur, nxt;
    memset(&cur, 0, sizeof(cur));
    lists_level0(vol, id_bytes, nx, ny, nz, &cur);
    g->max_nnz = 1;
    int64_t bufcap = 16;
    uint32_t *nbuf = (uint32_t *)malloc((size_t)bufcap * sizeof(uint32_t));
    uint64_t *wbuf = (uint64_t *)malloc((size_t)bufcap * sizeof(uint64_t));
    for (int l = 1; l < g->L; l++) {
        memset(&nxt, 0, sizeof(nxt));
        if (lists_next(&cur, &nxt)) { table_free(&t); mgo_graph_free(g); return NULL; }
        lists_free(&cur);
        cur = nxt;
        g->mip[l] = (uint32_t *)malloc((size_t)cur.nv * sizeof(uint32_t));
        for (int64_t v = 0; v < cur.nv; v++) {
            int64_t n = (int64_t)(cur.off[v + 1] - cur.off[v]);
            if (n > g->max_nnz) g->max_nnz = n;
            g->pairs += n - 1;
            if (n > bufcap) {
                bufcap = n;
                nbuf = (uint32_t *)realloc(nbuf, (size_t)bufcap * sizeof(uint32_t));
                wbuf = (uint64_t *)realloc(wbuf, (size_t)bufcap * sizeof(uint64_t));
            }
            int64_t root = factor_one(&t, cur.ids + cur.off[v], cur.cnt + cur.off[v], n, nbuf, wbuf);
            if (root < 0) { table_free(&t); mgo_graph_free(g); return NULL; }
            g->mip[l][v] = (uint32_t)root;
        }
    }
    lists_free(&cur);
    free(nbuf); free(wbuf);

    if (relabel(g, &t)) { table_free(&t); mgo_graph_free(g); return NULL; }
    for (int l = 1; l < g->L; l++) {
        int64_t nv = g->dims[3 * l] * g->dims[3 * l + 1] * g->dims[3 * l + 2];
        for (int64_t v = 0; v < nv; v++) g->mip[l][v] = (uint32_t)g->canon[g->mip[l][v]];
    }
    free(g->canon); g->canon = NULL;
    table_free(&t);
    return g;
}

/* Factorise M given mixtures (CSR lists sorted by id, integer weights) with
 * the same rule and numbering; roots[m] receives the canonical node of list m.
 * Used to run the paper's worked examples (Fig. 2-4) through the oracle. */
mgo_graph *mgo_factor_lists(const uint64_t *off, const uint32_t *ids, const uint64_t *cnt, int64_t M,
                            uint32_t S, uint32_t *roots)
{
    mgo_graph *g = (mgo_graph *)calloc(1, sizeof(mgo_graph));
    if (!g) return NULL;
    g->S = S;
    g->L = 0;
    mgo_table t;
    if (table_init(&t, S)) { free(g); return NULL; }
    int64_t cap = 1;
    for (int64_t m = 0; m < M; m++) {
        int64_t n = (int64_t)(off[m + 1] - off[m]);
        if (n > cap) cap = n;
    }
    uint32_t *nbuf = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
    uint64_t *wbuf = (uint64_t *)malloc((size_t)cap * sizeof(uint64_t));
    for (int64_t m = 0; m < M; m++) {
        int64_t n = (int64_t)(off[m + 1] - off[m]);
        int64_t r = factor_one(&t, ids + off[m], cnt + off[m], n, nbuf, wbuf);
        roots[m] = (uint32_t)r;
    }
    free(nbuf); free(wbuf);
    if (relabel(g, &t)) { table_free(&t); mgo_graph_free(g); return NULL; }
    for (int64_t m = 0; m < M; m++) roots[m] = (uint32_t)g->canon[roots[m]];
    free(g->canon); g->canon = NULL;
    table_free(&t);
    return g;
}

/* Sec. 3.4: topological level of every node of a node table whose nodes come
 * after their predecessors: sources 0, else max(level of p, level of q) + 1,
 * in one linear scan. */
void mgo_depths(const uint32_t *p, const uint32_t *q, int64_t N, uint32_t S, int32_t *depth)
{
    for (int64_t k = 0; k < N; k++) {
        if ((uint32_t)k < S) { depth[k] = 0; continue; }
        int32_t dp = depth[p[k]], dq = depth[q[k]];
        depth[k] = (dp > dq ? dp : dq) + 1;
    }
}

/* accessors for the Python wrapper */
int64_t mgo_graph_nodes(const mgo_graph *g) { return g->N; }
int mgo_graph_depth(const mgo_graph *g) { return g->D; }
int mgo_graph_levels(const mgo_graph *g) { return g->L; }
int64_t mgo_graph_max_nnz(const mgo_graph *g) { return g->max_nnz; }
int64_t mgo_graph_pairs(const mgo_graph *g) { return g->pairs; }
void mgo_graph_dims(const mgo_graph *g, int64_t *dims)
{
    memcpy(dims, g->dims, (size_t)g->L * 3 * sizeof(int64_t));
}
void mgo_graph_nodes_copy(const mgo_graph *g, uint32_t *p, uint32_t *q, uint64_t *a, uint64_t *b,
                          int32_t *depth)
{
    memcpy(p, g->p, (size_t)g->N * sizeof(uint32_t));
    memcpy(q, g->q, (size_t)g->N * sizeof(uint32_t));
    memcpy(a, g->a, (size_t)g->N * sizeof(uint64_t));
    memcpy(b, g->b, (size_t)g->N * sizeof(uint64_t));
    memcpy(depth, g->depth, (size_t)g->N * sizeof(int32_t));
}
void mgo_graph_buckets_copy(const mgo_graph *g, int64_t *off)
{
    memcpy(off, g->bucket, (size_t)(g->D + 2) * sizeof(int64_t));
}
void mgo_graph_mip_copy(const mgo_graph *g, int level, uint32_t *out)
{
    int64_t nv = g->dims[3 * level] * g->dims[3 * level + 1] * g->dims[3 * level + 2];
    memcpy(out, g->mip[level], (size_t)nv * sizeof(uint32_t));
}

/* ------------------------------------------------------------------------ */
/* Exact expansion of one node (Sec. 3.2: a node's mixture is given by its    */
/* tree of lerps).  Pushes the integer total T from `node` to the sources:    */
/* the predecessors of (p, q, a, b) receive T*a/(a+b) and T*b/(a+b).  Any     */
/* node table that represents integer mixtures keeps every division exact;    */
/* returns -1 when one is not.  out is a dense histogram of S counters.       */
/* ------------------------------------------------------------------------ */
int mgo_expand(const uint32_t *p, const uint32_t *q, const uint64_t *a, const uint64_t *b,
               uint32_t S, uint32_t node, uint64_t T, uint64_t *out)
{
    size_t cap = 64, n = 0;
    uint32_t *sn = (uint32_t *)malloc(cap * sizeof(uint32_t));
    uint64_t *sw = (uint64_t *)malloc(cap * sizeof(uint64_t));
    sn[n] = node; sw[n] = T; n++;
    int rc = 0;
    while (n) {
        n--;
        uint32_t k = sn[n];
        uint64_t w = sw[n];
        if (k < S) { out[k] += w; continue; }
        uint64_t s = a[k] + b[k];
        if (s == 0 || w % s) { rc = -1; break; }
        uint64_t t = w / s;
        if (n + 2 > cap) {
            cap *= 2;
            sn = (uint32_t *)realloc(sn, cap * sizeof(uint32_t));
            sw = (uint64_t *)realloc(sw, cap * sizeof(uint64_t));
        }
        sn[n] = p[k]; sw[n] = t * a[k]; n++;
        sn[n] = q[k]; sw[n] = t * b[k]; n++;
    }
    free(sn); free(sw);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 / Sec. 4: colour propagation over the node table in topological   */
/* (ID) order, fp64: val[s] = TF[s]; val[n] = (a*val[p] + b*val[q])/(a+b).    */
/* ------------------------------------------------------------------------ */
void mgo_propagate(const uint32_t *p, const uint32_t *q, const uint64_t *a, const uint64_t *b,
                   int64_t N, uint32_t S, const double *tf, int C, double *val)
{
    for (uint32_t s = 0; s < S; s++)
        for (int c = 0; c < C; c++) val[(int64_t)s * C + c] = tf[(int64_t)s * C + c];
    for (int64_t k = S; k < N; k++) {
        double wa = (double)a[k], wb = (double)b[k];
        for (int c = 0; c < C; c++)
            val[k * C + c] = (wa * val[(int64_t)p[k] * C + c] + wb * val[(int64_t)q[k] * C + c]) / (wa + wb);
    }
}

/* Direct colour of every voxel of one level: sum_i H_i * TF(i), fp64, from
 * the integer mixture lists (count / 8^l). */
void mgo_direct_colors(const uint64_t *off, const uint32_t *ids, const uint64_t *cnt, int64_t nv,
                       const double *tf, int C, double *out)
{
    for (int64_t v = 0; v < nv; v++) {
        uint64_t tot = 0;
        for (uint64_t e = off[v]; e < off[v + 1]; e++) tot += cnt[e];
        for (int c = 0; c < C; c++) {
            double s = 0.0;
            for (uint64_t e = off[v]; e < off[v + 1]; e++)
                s += (double)cnt[e] * tf[(int64_t)ids[e] * C + c];
            out[v * C + c] = s / (double)tot;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Box histogram by brute force (the plain definition of a sub-volume query, */
/* Sec. 3.6): count the level-0 IDs inside the box clipped to the volume.    */
/* Box = (x, y, z, dx, dy, dz); out is Q x S, zeroed here.                   */
/* ------------------------------------------------------------------------ */
void mgo_box_hist(const void *vol, int id_bytes, int64_t nx, int64_t ny, int64_t nz, uint32_t S,
                  const int32_t *boxes, int64_t Q, uint32_t *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t qi = 0; qi < Q; qi++) {
        const int32_t *bx = boxes + 6 * qi;
        uint32_t *h = out + qi * (int64_t)S;
        for (uint32_t s = 0; s < S; s++) h[s] = 0;
        int64_t x1 = bx[0] + (int64_t)bx[3]; if (x1 > nx) x1 = nx;
        int64_t y1 = bx[1] + (int64_t)bx[4]; if (y1 > ny) y1 = ny;
        int64_t z1 = bx[2] + (int64_t)bx[5]; if (z1 > nz) z1 = nz;
        for (int64_t z = bx[2]; z < z1; z++)
            for (int64_t y = bx[1]; y < y1; y++)
                for (int64_t x = bx[0]; x < x1; x++)
                    h[vol_id(vol, id_bytes, (z * ny + y) * nx + x)]++;
    }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Sec. 3.6): footprint assembly.                               */
/* ------------------------------------------------------------------------ */
static int floor_log2_u64(uint64_t x)
{
    int r = -1;
    while (x) { x >>= 1; r++; }
    return r;
}

static int ctz_or_inf(uint64_t x)
{
    if (x == 0) return 1000;          /* tzcnt(0) is taken as infinite (R6) */
    int r = 0;
    while (!(x & 1)) { x >>= 1; r++; }
    return r;
}

/* footprint_1d: aligned power-of-two steps covering [i, i+di) clipped to dim */
int mgo_footprint_1d(int64_t i, int64_t di, int64_t dim, int32_t *r)
{
    int n = 0;
    di = ((i + di) < dim ? (i + di) : dim) - i;
    while (di > 0) {
        int a = floor_log2_u64((uint64_t)di);
        int b = ctz_or_inf((uint64_t)i);
        int l = a < b ? a : b;
        r[n++] = l;
        di -= (int64_t)1 << l;
        i += (int64_t)1 << l;
    }
    return n;
}

/* Enumerate the cubes of one box: for every cube, its level and level-l voxel
 * coordinates.  Returns the number of cubes; writes at most `cap` of them
 * (cubes may be NULL to only count). */
int64_t mgo_fa_cubes(const int32_t *box, int64_t nx, int64_t ny, int64_t nz,
                     int32_t *cubes /* 4 per cube: l, x, y, z */, int64_t cap)
{
    int32_t Lx[80], Ly[80], Lz[80];
    int nxr = mgo_footprint_1d(box[0], box[3], nx, Lx);
    int nyr = mgo_footprint_1d(box[1], box[4], ny, Ly);
    int nzr = mgo_footprint_1d(box[2], box[5], nz, Lz);
    int64_t qx, qy, qz = box[2];
    int64_t n = 0;
    for (int k = 0; k < nzr; k++) {
        qy = box[1];
        for (int j = 0; j < nyr; j++) {
            qx = box[0];
            for (int i = 0; i < nxr; i++) {
                int l = Lx[i];
                if (Ly[j] < l) l = Ly[j];
                if (Lz[k] < l) l = Lz[k];
                int64_t ex = (int64_t)1 << (Lx[i] - l);
                int64_t ey = (int64_t)1 << (Ly[j] - l);
                int64_t ez = (int64_t)1 << (Lz[k] - l);
                for (int64_t w = 0; w < ez; w++)
                    for (int64_t v = 0; v < ey; v++)
                        for (int64_t u = 0; u < ex; u++) {
                            if (cubes && n < cap) {
                                cubes[4 * n + 0] = l;
                                cubes[4 * n + 1] = (int32_t)((qx >> l) + u);
                                cubes[4 * n + 2] = (int32_t)((qy >> l) + v);
                                cubes[4 * n + 3] = (int32_t)((qz >> l) + w);
                            }
                            n++;
                        }
                qx += (int64_t)1 << Lx[i];
            }
            qy += (int64_t)1 << Ly[j];
        }
        qz += (int64_t)1 << Lz[k];
    }
    return n;
}

/* Box histogram by footprint assembly over an oracle graph: every cube at
 * level l contributes 8^l through its mip node, pushed exactly to the sources.
 * Returns -1 if an inexact division is met.  out is Q x S, zeroed here. */
int mgo_fa_query(const mgo_graph *g, const int32_t *boxes, int64_t Q, uint32_t *out)
{
    uint32_t S = g->S;
    uint64_t *acc = (uint64_t *)malloc((size_t)S * sizeof(uint64_t));
    int rc = 0;
    for (int64_t qi = 0; qi < Q && rc == 0; qi++) {
        const int32_t *bx = boxes + 6 * qi;
        memset(acc, 0, (size_t)S * sizeof(uint64_t));
        int64_t nc = mgo_fa_cubes(bx, g->dims[0], g->dims[1], g->dims[2], NULL, 0);
        int32_t *cubes = (int32_t *)malloc((size_t)(nc > 0 ? nc : 1) * 4 * sizeof(int32_t));
        mgo_fa_cubes(bx, g->dims[0], g->dims[1], g->dims[2], cubes, nc);
        for (int64_t c = 0; c < nc && rc == 0; c++) {
            int l = cubes[4 * c];
            const int64_t *dl = g->dims + 3 * l;
            int64_t v = ((int64_t)cubes[4 * c + 3] * dl[1] + cubes[4 * c + 2]) * dl[0] + cubes[4 * c + 1];
            uint64_t w = (uint64_t)1 << (3 * l);
            rc = mgo_expand(g->p, g->q, g->a, g->b, S, g->mip[l][v], w, acc);
        }
        free(cubes);
        for (uint32_t s = 0; s < S; s++) out[qi * (int64_t)S + s] = (uint32_t)acc[s];
    }
    free(acc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Ray-sample lookup (Sec. 4): nearest voxel of the level nearest to the     */
/* sample's LOD.  The level and voxel index are decided in fp32, the           */
/* precision of the samples.  Sample = (x, y, z, lod) in level-0 voxel units. */
/* ------------------------------------------------------------------------ */
static int64_t floor_coord(float x, int64_t d0)
{
    /* clamp to [0, d0] in fp32 (NaN goes to 0), then floor; for x >= 0 the
     * truncating conversion is the floor */
    float xc = x;
    if (!(xc >= 0.0f)) xc = 0.0f;
    if (xc > (float)d0) xc = (float)d0;
    return (int64_t)xc;
}

static int sample_level(float lod, int L)
{
    float t = lod + 0.5f;               /* round to the nearest level, fp32 */
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)(L - 1)) return L - 1;
    return (int)t;
}

/* For every sample: its level and the linear index of its voxel in that
 * level (x fastest). */
void mgo_sample_voxels(const int64_t *dims, int L, const float *samples, int64_t P,
                       int32_t *level_out, int64_t *voxel_out)
{
    for (int64_t i = 0; i < P; i++) {
        const float *s = samples + 4 * i;
        int l = sample_level(s[3], L);
        const int64_t *dl = dims + 3 * l;
        int64_t v[3];
        for (int k = 0; k < 3; k++) {
            int64_t c = floor_coord(s[k], dims[k]) >> l;
            v[k] = c < dl[k] - 1 ? c : dl[k] - 1;
        }
        level_out[i] = l;
        voxel_out[i] = (v[2] * dl[1] + v[1]) * dl[0] + v[0];
    }
}

/* Threads of the OpenMP loops (box counting); returns the number now in use.
 * Used to report the baseline both single-threaded and on all cores. */
int mgo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sec. 4: ray marching through the palette of node values.                  */
/*                                                                          */
/* Readings taken here (Sec. 4 names the parts, not their formulas):         */
/*   F1 the LOD of a sample is floor(log2(t * pixel angle)) + bias (pixel     */
/*      coverage linear in depth); it picks mip level m = clamp(LOD, 0, L-1) */
/*      and the step: samples lie on the lattice t_k = t_start + k * base,    */
/*      and a sample at level m advances k by 2^m (step adjusted to the LOD). */
/*   F2 "interpolation ... manually": trilinear within level m between the    */
/*      8 voxel centres around the sample (clamped to the level), and        */
/*      linear between levels m and m+1 by the fractional LOD (quadrilinear).*/
/*   F3 opacity correction for a step of 2^e base steps:                     */
/*      alpha' = 1 - (1 - alpha)^(2^e); front-to-back compositing of the    */
/*      sample's colour with weight (1 - A) * alpha'; the ray stops once A   */
/*      reaches the early-termination opacity.                               */
/*   F4 empty-space skipping: opacities propagated through the graph (the    */
/*      mixture average of the TF's alpha) give every mip voxel's opacity;   */
/*      climbing from level m+2 while the voxel around the sample has       */
/*      opacity exactly 0, the largest such voxel, shrunk by 3 * 2^m on      */
/*      every side (the reach of the sample's interpolation), is skipped:    */
/*      the lattice samples inside it and before the next LOD change would   */
/*      each add exactly nothing.                                            */
/* Every decision (lattice position, level, skip, termination) is taken in   */
/* fp32 with one rounding per operation, the precision of the GPU path.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    float eye[3], fwd[3], right[3], up[3];
    float pix;
    int32_t width, height;
    float base_step;
    int32_t lod_bias;
    float ert;
    int32_t max_steps;
    int32_t reserved[4];
} mgo_camera;

static float rm_lerp(float a, float b, float f) { return a + f * (b - a); }

static uint32_t rm_node(const mgo_graph *g, int l, int64_t x, int64_t y, int64_t z)
{
    const int64_t *d = g->dims + 3 * l;
    return g->mip[l][(z * d[1] + y) * d[0] + x];
}

/* trilinear value (4 channels) of level l at position p (level-0 units) */
static void rm_tri(const mgo_graph *g, const float *vals, int l, const float *p, float *out)
{
    const int64_t *d = g->dims + 3 * l;
    float scale = ldexpf(1.0f, -l);
    int64_t i0[3], i1[3];
    float f[3];
    for (int c = 0; c < 3; c++) {
        float u = p[c] * scale - 0.5f;
        float fl = floorf(u);
        f[c] = u - fl;
        int64_t k = (int64_t)fl;
        i0[c] = k < 0 ? 0 : (k > d[c] - 1 ? d[c] - 1 : k);
        i1[c] = k + 1 < 0 ? 0 : (k + 1 > d[c] - 1 ? d[c] - 1 : k + 1);
    }
    float v[8][4];
    for (int corner = 0; corner < 8; corner++) {
        int64_t x = corner & 1 ? i1[0] : i0[0], y = corner & 2 ? i1[1] : i0[1], z = corner & 4 ? i1[2] : i0[2];
        const float *r = vals + 4 * (int64_t)rm_node(g, l, x, y, z);
        for (int ch = 0; ch < 4; ch++) v[corner][ch] = r[ch];
    }
    for (int ch = 0; ch < 4; ch++) {
        float x00 = rm_lerp(v[0][ch], v[1][ch], f[0]), x10 = rm_lerp(v[2][ch], v[3][ch], f[0]);
        float x01 = rm_lerp(v[4][ch], v[5][ch], f[0]), x11 = rm_lerp(v[6][ch], v[7][ch], f[0]);
        float y0 = rm_lerp(x00, x10, f[1]), y1 = rm_lerp(x01, x11, f[1]);
        out[ch] = rm_lerp(y0, y1, f[2]);
    }
}

/* One image of width x height RGBA (fp32, row 0 at the top).  vals: N x 4
 * node values; opac: N node opacities (NULL: no skipping).  steps_out (may
 * be NULL): samples composited per pixel; margin_out (may be NULL): the
 * smallest |A - ert| seen after a sample (+inf when ert > 1). */
void mgo_raymarch(const mgo_graph *g, const float *vals, const float *opac, const mgo_camera *cam, float *img,
                  int32_t *steps_out, float *margin_out)
{
    const int L = g->L;
    const int W = cam->width, H = cam->height;
    const float inf = 3.0e38f;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t pix_i = 0; pix_i < (int64_t)W * H; pix_i++) {
        int i = (int)(pix_i % W), j = (int)(pix_i / W);
        float sx = (((float)i + 0.5f) - 0.5f * (float)W) * cam->pix;
        float sy = ((0.5f * (float)H - (float)j) - 0.5f) * cam->pix;
        float d[3];
        for (int c = 0; c < 3; c++) d[c] = (cam->fwd[c] + sx * cam->right[c]) + sy * cam->up[c];
        float nrm = sqrtf((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
        for (int c = 0; c < 3; c++) d[c] = d[c] / nrm;
        float tmin = -inf, tmax = inf;
        int miss = 0;
        for (int c = 0; c < 3; c++) {
            float dim = (float)g->dims[c];
            if (d[c] == 0.0f) {
                if (cam->eye[c] < 0.0f || cam->eye[c] > dim) miss = 1;
                continue;
            }
            float t0 = (0.0f - cam->eye[c]) / d[c], t1 = (dim - cam->eye[c]) / d[c];
            float lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
            if (lo > tmin) tmin = lo;
            if (hi < tmax) tmax = hi;
        }
        float ts = tmin > 0.0f ? tmin : 0.0f;
        float C[3] = {0.0f, 0.0f, 0.0f}, A = 0.0f, margin = inf;
        int32_t taken = 0;
        if (!miss && tmax > ts) {
            int64_t k = 0;
            while (k < cam->max_steps) {
                float t = ts + (float)k * cam->base_step;
                if (!(t < tmax)) break;
                float x = t * cam->pix;
                int lam = x > 0.0f ? ilogbf(x) + cam->lod_bias : -1000000;
                int m = lam < 0 ? 0 : (lam > L - 1 ? L - 1 : lam);
                float fr = 0.0f;
                if (lam >= 0 && m < L - 1) {
                    fr = (log2f(x) + (float)cam->lod_bias) - (float)lam;
                    fr = fr < 0.0f ? 0.0f : (fr > 1.0f ? 1.0f : fr);
                }
                float p[3];
                for (int c = 0; c < 3; c++) p[c] = cam->eye[c] + t * d[c];
                if (opac) {
                    int jz = -1;
                    int64_t bz[3] = {0, 0, 0};
                    for (int jl = m + 2; jl < L; jl++) {
                        int64_t b[3];
                        for (int c = 0; c < 3; c++) {
                            int64_t v = (int64_t)floorf(p[c]);
                            v = v < 0 ? 0 : v;
                            v >>= jl;
                            b[c] = v > g->dims[3 * jl + c] - 1 ? g->dims[3 * jl + c] - 1 : v;
                        }
                        if (opac[rm_node(g, jl, b[0], b[1], b[2])] != 0.0f) break;
                        jz = jl;
                        for (int c = 0; c < 3; c++) bz[c] = b[c];
                    }
                    if (jz >= 0) {
                        float size = ldexpf(1.0f, jz), gap = ldexpf(3.0f, m);
                        float lo[3], hi[3];
                        int inside = 1;
                        for (int c = 0; c < 3; c++) {
                            lo[c] = (float)bz[c] * size + gap;
                            hi[c] = ((float)bz[c] + 1.0f) * size - gap;
                            if (!(p[c] > lo[c] && p[c] < hi[c])) inside = 0;
                        }
                        if (inside) {
                            float tout = inf;
                            for (int c = 0; c < 3; c++) {
                                float te = d[c] > 0.0f ? (hi[c] - cam->eye[c]) / d[c]
                                                       : d[c] < 0.0f ? (lo[c] - cam->eye[c]) / d[c] : inf;
                                if (te < tout) tout = te;
                            }
                            float tch = m < L - 1 ? ldexpf(1.0f, lam + 1 - cam->lod_bias) / cam->pix : inf;
                            float tl = tout < tch ? tout : tch;
                            float len = (float)((int64_t)1 << m) * cam->base_step;
                            int64_t n = (int64_t)floorf((tl - t) / len) - 1;
                            if (n >= 1) {
                                k += n << m;
                                continue;
                            }
                        }
                    }
                }
                float s[4], s1[4];
                rm_tri(g, vals, m, p, s);
                if (fr > 0.0f) {
                    rm_tri(g, vals, m + 1, p, s1);
                    for (int ch = 0; ch < 4; ch++) s[ch] = rm_lerp(s[ch], s1[ch], fr);
                }
                float q = 1.0f - s[3];
                for (int e = 0; e < m; e++) q = q * q;
                float ap = 1.0f - q;
                float w = (1.0f - A) * ap;
                for (int c = 0; c < 3; c++) C[c] = C[c] + w * s[c];
                A = A + w;
                taken++;
                if (cam->ert <= 1.0f) {
                    float dm = A > cam->ert ? A - cam->ert : cam->ert - A;
                    if (dm < margin) margin = dm;
                    if (A >= cam->ert) break;
                }
                k += (int64_t)1 << m;
            }
        }
        float *o = img + 4 * pix_i;
        o[0] = C[0]; o[1] = C[1]; o[2] = C[2]; o[3] = A;
        if (steps_out) steps_out[pix_i] = taken;
        if (margin_out) margin_out[pix_i] = margin;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3, Table 1, Eq. 14-15: the bitstream of a graph.                   */
/*                                                                          */
/* Readings taken here:                                                      */
/*   B1 bit order: every field is written least significant bit first, and  */
/*      bit i of the stream is bit (i mod 8) of byte i / 8.                  */
/*   B2 ranges [1..64] and [1..16] (fields (3) and (6)) are stored minus one.*/
/*   B3 Table 1 has no lossless form: the exact graph's weights a:b (no     */
/*      quantiser) go into an extension after field (7): one bit "exact"    */
/*      (1 here) and six bits holding w - 1, w the width of the larger of a  */
/*      and b; then every node of (B) stores p, q at field (3)'s width and   */
/*      a, b at w bits instead of a codebook index, and (C) is empty.  Field */
/*      (6) holds 1 and field (4) holds 0.                                   */
/*   B4 field (3) is ceil(log2 N) (at least 1); field (7) is N - S; levels   */
/*      go from 0 (the input) to L - 1, and (A) lists each level's voxels    */
/*      x fastest, as ID - i_min(l) at r(l) = ceil(log2(i_max - i_min + 1))  */
/*      bits (Eq. 15; 0 bits when the level holds one ID).                   */
/*   B5 the stream is padded with zero bytes to a multiple of 8 bytes.       */
/* ------------------------------------------------------------------------ */
typedef struct { uint8_t *buf; int64_t cap; int64_t bit; } bs_writer;

static void bs_put(bs_writer *w, uint64_t v, int nbits)
{
    for (int i = 0; i < nbits; i++) {
        if ((v >> i) & 1u) {
            int64_t byte = (w->bit + i) >> 3;
            if (byte < w->cap) w->buf[byte] |= (uint8_t)(1u << ((w->bit + i) & 7));
        }
    }
    w->bit += nbits;
}

static int bits_for(uint64_t range)   /* ceil(log2(range)), range >= 1 */
{
    int b = 0;
    while (b < 64 && ((uint64_t)1 << b) < range) b++;
    return b;
}

/* Writes the stream into out (cap bytes, zeroed here); returns its size in
 * bytes (call with out = NULL for the size alone). */
int64_t mgo_bitstream(const mgo_graph *g, uint8_t *out, int64_t cap)
{
    int nb = bits_for((uint64_t)g->N);
    if (nb < 1) nb = 1;
    uint64_t wmax = 1;
    for (int64_t n = g->S; n < g->N; n++) {
        if (g->a[n] > wmax) wmax = g->a[n];
        if (g->b[n] > wmax) wmax = g->b[n];
    }
    int wbits = bits_for(wmax + 1);
    if (wbits < 1) wbits = 1;
    uint32_t imin[MGO_MAX_LEVELS], rl[MGO_MAX_LEVELS];
    for (int l = 0; l < g->L; l++) {
        int64_t nv = g->dims[3 * l] * g->dims[3 * l + 1] * g->dims[3 * l + 2];
        uint32_t lo = g->mip[l][0], hi = g->mip[l][0];
        for (int64_t v = 1; v < nv; v++) {
            if (g->mip[l][v] < lo) lo = g->mip[l][v];
            if (g->mip[l][v] > hi) hi = g->mip[l][v];
        }
        imin[l] = lo;
        rl[l] = (uint32_t)bits_for((uint64_t)(hi - lo) + 1);
    }
    bs_writer w = {out, out ? cap : 0, 0};
    if (out) memset(out, 0, (size_t)cap);
    bs_put(&w, g->S, 32);                       /* (1) sources */
    bs_put(&w, 0, 1);                           /* (2) fractional input: no */
    bs_put(&w, (uint64_t)(nb - 1), 6);          /* (3) bits per node */
    bs_put(&w, 0, 32);                          /* (4) sigma_max (no quantiser) */
    for (int k = 0; k < 3; k++) bs_put(&w, (uint64_t)g->dims[k], 32);   /* (5) resolution */
    bs_put(&w, 0, 4);                           /* (6) quantisation bitrate 1 (unused) */
    bs_put(&w, (uint64_t)(g->N - g->S), nb);    /* (7) internal nodes */
    bs_put(&w, 1, 1);                           /* extension: exact weights */
    bs_put(&w, (uint64_t)(wbits - 1), 6);       /*            their width */
    for (int l = 0; l < g->L; l++) {
        bs_put(&w, rl[l], nb);                  /* (8) voxel bits */
        bs_put(&w, imin[l], nb);                /* (9) i_min(l) */
    }
    for (int l = 0; l < g->L; l++) {           /* (A) one mixture ID per voxel */
        int64_t nv = g->dims[3 * l] * g->dims[3 * l + 1] * g->dims[3 * l + 2];
        for (int64_t v = 0; v < nv; v++) bs_put(&w, g->mip[l][v] - imin[l], (int)rl[l]);
    }
    for (int64_t n = g->S; n < g->N; n++) {    /* (B) description of mixtures */
        bs_put(&w, g->p[n], nb);
        bs_put(&w, g->q[n], nb);
        bs_put(&w, g->a[n], wbits);
        bs_put(&w, g->b[n], wbits);
    }
    int64_t bytes = (w.bit + 7) >> 3;
    return (bytes + 7) & ~(int64_t)7;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3 (Eq. 10-13) and Sec. 3.7: greedy factorisation.                  */
/*                                                                          */
/* Readings taken here:                                                      */
/*   G1 H is every mixture of levels 1..L-1 (level-0 voxels are sources).   */
/*      Components are node IDs with exact integer weights (8^l H, R1).     */
/*   G2 stage 1 (Sec. 3.7): only mixtures with more than tau components are */
/*      scored and factored.  A round scores every pair i < j of components */
/*      that occur together in such a mixture h, phi_1 adding 1 per h and   */
/*      phi_2 adding |h| - 1 if |h| > 2, else 2 (Eq. 10-13); the pick is the */
/*      highest score, ties to the smallest (i, j); every such mixture that */
/*      holds both is factored (all occurrences).  Stage 1 ends when no      */
/*      mixture has more than tau components.                               */
/*   G3 stage 2: the mixtures left with 2..tau components are factorised in */
/*      waves: in each, every such mixture, levels in order and voxels x     */
/*      fastest, lerps its two lowest-numbered components.  Nodes are        */
/*      numbered in order of creation, so a wave's new nodes follow the scan */
/*      position of the first mixture that made them (as a parallel build   */
/*      numbers them).                                                       */
/*   G4 a lerp of components p < q with weights c_p, c_q gives q the weight */
/*      w = c_q / (c_p + c_q).  bitrate b >= 1: w falls in bin k = floor(w   */
/*      2^b) of the 2^b equal bins of (0, 1), decided exactly in integers;   */
/*      the node is the key (p, q, k), so all lerps of one pair in one bin   */
/*      are one node; the bin's codeword is its centre (2k + 1) / 2^(b+1)    */
/*      and its sigma the rms of w - codeword over the lerps in the bin.     */
/*      The bins are symmetric about 1/2, so the symmetry of Sec. 3.7         */
/*      ((i, j, w) = (j, i, 1 - w)) never lowers the error: orientation p<q.*/
/*      b = 0: exact, the node is the key (p, q, a, b) of the reduced ratio  */
/*      a:b = c_p:c_q as in the pairwise graph.                              */
/*   G5 the merged component keeps the exact weight c_p + c_q.  Node IDs are */
/*      canonical (R5); a quantised node holds its bin in `a` and 0 in `b`.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t M;            /* mixtures (levels 1..L-1, level by level, x fastest) */
    int64_t *off;         /* first entry of every mixture (M + 1) */
    int32_t *len;         /* current number of components */
    uint32_t *comp;       /* component node IDs, ascending within a mixture */
    uint64_t *wt;         /* their exact weights */
} gr_lists;

static void gr_free(gr_lists *x)
{
    free(x->off); free(x->len); free(x->comp); free(x->wt);
    memset(x, 0, sizeof(*x));
}

/* lerp of (p, cp), (q, cq), p < q: the node, and the quantiser's record */
static int64_t gr_node(mgo_table *t, uint32_t p, uint64_t cp, uint32_t q, uint64_t cq, int bitrate,
                       double *ssq, int64_t *cnt)
{
    if (bitrate == 0) return table_get(t, p, cp, q, cq);
    uint64_t s = cp + cq;
    uint64_t k = (cq << bitrate) / s;      /* floor(w 2^b), w in (0, 1) */
    uint64_t nb = (uint64_t)1 << bitrate;
    if (k >= nb) k = nb - 1;
    double w = (double)cq / (double)s, c = ((double)(2 * k + 1)) / (double)(2 * nb);
    ssq[k] += (w - c) * (w - c);
    cnt[k]++;
    return table_get_key(t, p, q, k, 0);
}

/* replace components i, j (both present, i < j) of mixture m by node n with
 * weight ci + cj, keeping the list ascending */
static void gr_merge(gr_lists *x, int64_t m, int32_t ii, int32_t jj, uint32_t n, uint64_t w)
{
    uint32_t *c = x->comp + x->off[m];
    uint64_t *v = x->wt + x->off[m];
    int32_t L = x->len[m], o = 0;
    for (int32_t e = 0; e < L; e++) {
        if (e == ii || e == jj) continue;
        c[o] = c[e]; v[o] = v[e]; o++;
    }
    int32_t pos = o;
    while (pos > 0 && c[pos - 1] > n) { c[pos] = c[pos - 1]; v[pos] = v[pos - 1]; pos--; }
    c[pos] = n; v[pos] = w;
    x->len[m] = o + 1;
}

static int32_t gr_find(const gr_lists *x, int64_t m, uint32_t id)
{
    const uint32_t *c = x->comp + x->off[m];
    int32_t lo = 0, hi = x->len[m];
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (c[mid] < id) lo = mid + 1; else hi = mid;
    }
    return lo < x->len[m] && c[lo] == id ? lo : -1;
}

typedef struct { uint32_t i, j; uint64_t score; int used; } gr_pair;

/* Stages 1 and 2 on the mixtures x (G2, G3), nodes into t; the quantiser's
 * records into ssq / cnt; the stage-1 picks into picks (room for max_picks). */
static void gr_run(gr_lists *x, mgo_table *t, int strategy, int tau, int bitrate, double *ssq, int64_t *cnt,
                   uint32_t *picks, int64_t max_picks, int64_t *n_picks)
{
    int64_t npick = 0;
    const int64_t M = x->M;

    /* stage 1: greedy picks over the mixtures with more than tau components */
    int64_t pcap = 1024, pn = 0;
    gr_pair *pairs = (gr_pair *)malloc((size_t)pcap * sizeof(gr_pair));
    int64_t hcap = 1;
    int64_t *hslot = NULL;
    for (;;) {
        /* scores: an open-addressing map (i, j) -> index into pairs */
        pn = 0;
        int64_t need = 16;
        for (int64_t m = 0; m < M; m++)
            if (x->len[m] > tau) need += (int64_t)x->len[m] * (x->len[m] - 1) / 2;
        if (need <= 16) break;
        while (hcap < 2 * need) hcap *= 2;
        hslot = (int64_t *)realloc(hslot, (size_t)hcap * sizeof(int64_t));
        for (int64_t i = 0; i < hcap; i++) hslot[i] = -1;
        for (int64_t m = 0; m < M; m++) {
            int32_t n = x->len[m];
            if (n <= tau) continue;
            uint64_t add = strategy == 1 ? 1 : (n > 2 ? (uint64_t)(n - 1) : 2);
            const uint32_t *c = x->comp + x->off[m];
            for (int32_t a = 0; a < n; a++)
                for (int32_t b2 = a + 1; b2 < n; b2++) {
                    uint64_t h = mix64(((uint64_t)c[a] << 32) | c[b2]) & (uint64_t)(hcap - 1);
                    while (hslot[h] >= 0 && !(pairs[hslot[h]].i == c[a] && pairs[hslot[h]].j == c[b2]))
                        h = (h + 1) & (uint64_t)(hcap - 1);
                    if (hslot[h] < 0) {
                        if (pn == pcap) { pcap *= 2; pairs = (gr_pair *)realloc(pairs, (size_t)pcap * sizeof(gr_pair)); }
                        pairs[pn].i = c[a]; pairs[pn].j = c[b2]; pairs[pn].score = 0;
                        hslot[h] = pn++;
                    }
                    pairs[hslot[h]].score += add;
                }
        }
        int64_t best = -1;
        for (int64_t k = 0; k < pn; k++) {
            if (best < 0 || pairs[k].score > pairs[best].score ||
                (pairs[k].score == pairs[best].score &&
                 (pairs[k].i < pairs[best].i || (pairs[k].i == pairs[best].i && pairs[k].j < pairs[best].j))))
                best = k;
        }
        if (best < 0) break;
        uint32_t bi = pairs[best].i, bj = pairs[best].j;
        if (picks && npick < max_picks) { picks[2 * npick] = bi; picks[2 * npick + 1] = bj; }
        npick++;
        /* factor every occurrence among the mixtures with more than tau components */
        for (int64_t m = 0; m < M; m++) {
            if (x->len[m] <= tau) continue;
            int32_t ii = gr_find(x, m, bi), jj = gr_find(x, m, bj);
            if (ii < 0 || jj < 0) continue;
            uint64_t ci = x->wt[x->off[m] + ii], cj = x->wt[x->off[m] + jj];
            int64_t nd = gr_node(t, bi, ci, bj, cj, bitrate, ssq, cnt);
            gr_merge(x, m, ii, jj, (uint32_t)nd, ci + cj);
        }
    }
    free(pairs); free(hslot);

    /* stage 2: waves over the rest in scanline order, each mixture lerping
     * its two lowest components per wave */
    for (int any = 1; any;) {
        any = 0;
        for (int64_t m = 0; m < M; m++) {
            if (x->len[m] < 2) continue;
            const uint32_t *c = x->comp + x->off[m];
            uint32_t p = c[0], q = c[1];
            uint64_t cp = x->wt[x->off[m]], cq = x->wt[x->off[m] + 1];
            int64_t nd = gr_node(t, p, cp, q, cq, bitrate, ssq, cnt);
            gr_merge(x, m, 0, 1, (uint32_t)nd, cp + cq);
            any = 1;
        }
    }

    *n_picks = npick;
}

/* The greedy graph of a volume; codebook / sigma (2^bitrate each, may be
 * NULL) receive the codewords and rms errors, picks (may be NULL, room for
 * max_picks pairs) the stage-1 picks in order, *n_picks their number. */
mgo_graph *mgo_build_greedy(const void *vol, int id_bytes, int64_t nx, int64_t ny, int64_t nz, uint32_t S,
                            int strategy, int tau, int bitrate, double *codebook, double *sigma,
                            uint32_t *picks, int64_t max_picks, int64_t *n_picks)
{
    if (strategy != 1 && strategy != 2) return NULL;
    if (bitrate < 0 || bitrate > 16 || tau < 1) return NULL;
    mgo_graph *g = (mgo_graph *)calloc(1, sizeof(mgo_graph));
    if (!g) return NULL;
    g->S = S;
    g->L = mgo_level_dims(nx, ny, nz, g->dims, MGO_MAX_LEVELS);
    int64_t V0 = nx * ny * nz;
    for (int64_t i = 0; i < V0; i++) if (vol_id(vol, id_bytes, i) >= S) { free(g); return NULL; }
    g->mip = (uint32_t **)calloc((size_t)g->L, sizeof(uint32_t *));
    g->mip[0] = (uint32_t *)malloc((size_t)V0 * sizeof(uint32_t));
    for (int64_t i = 0; i < V0; i++) g->mip[0][i] = vol_id(vol, id_bytes, i);

    /* H: the mixtures of levels 1..L-1 */
    int64_t M = 0, E = 0;
    mgo_lists lv[MGO_MAX_LEVELS];
    memset(lv, 0, sizeof(lv));
    lists_level0(vol, id_bytes, nx, ny, nz, &lv[0]);
    for (int l = 1; l < g->L; l++) {
        if (lists_next(&lv[l - 1], &lv[l])) {
            for (int k = 0; k <= l; k++) lists_free(&lv[k]);
            mgo_graph_free(g);
            return NULL;
        }
        if (l == 1) lists_free(&lv[0]);
        M += lv[l].nv;
        E += lv[l].nnz;
    }
    if (g->L == 1) lists_free(&lv[0]);
    gr_lists x;
    x.M = M;
    x.off = (int64_t *)malloc((size_t)(M + 1) * sizeof(int64_t));
    x.len = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    x.comp = (uint32_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(uint32_t));
    x.wt = (uint64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(uint64_t));
    {
        int64_t m = 0, e = 0;
        for (int l = 1; l < g->L; l++) {
            for (int64_t v = 0; v < lv[l].nv; v++, m++) {
                x.off[m] = e;
                x.len[m] = (int32_t)(lv[l].off[v + 1] - lv[l].off[v]);
                for (uint64_t k = lv[l].off[v]; k < lv[l].off[v + 1]; k++, e++) {
                    x.comp[e] = lv[l].ids[k];
                    x.wt[e] = lv[l].cnt[k];
                }
            }
            if (lv[l].nv) {
                int64_t nv = lv[l].nv;
                for (int64_t v = 0; v < nv; v++) {
                    int64_t n = (int64_t)(lv[l].off[v + 1] - lv[l].off[v]);
                    if (n > g->max_nnz) g->max_nnz = n;
                    g->pairs += n - 1;
                }
            }
            lists_free(&lv[l]);
        }
        x.off[M] = e;
    }
    if (g->max_nnz < 1) g->max_nnz = 1;

    mgo_table t;
    table_init(&t, S);
    int64_t nbins = bitrate ? ((int64_t)1 << bitrate) : 1;
    double *ssq = (double *)calloc((size_t)nbins, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nbins, sizeof(int64_t));
    int64_t npick = 0;
    gr_run(&x, &t, strategy, tau, bitrate, ssq, cnt, picks, max_picks, &npick);

    /* mip IDs (temporary numbers), then the canonical numbering */
    {
        int64_t m = 0;
        for (int l = 1; l < g->L; l++) {
            int64_t nv = g->dims[3 * l] * g->dims[3 * l + 1] * g->dims[3 * l + 2];
            g->mip[l] = (uint32_t *)malloc((size_t)nv * sizeof(uint32_t));
            for (int64_t v = 0; v < nv; v++, m++) g->mip[l][v] = x.comp[x.off[m]];
        }
    }
    gr_free(&x);
    if (relabel(g, &t)) { table_free(&t); mgo_graph_free(g); free(ssq); free(cnt); return NULL; }
    for (int l = 1; l < g->L; l++) {
        int64_t nv = g->dims[3 * l] * g->dims[3 * l + 1] * g->dims[3 * l + 2];
        for (int64_t v = 0; v < nv; v++) g->mip[l][v] = (uint32_t)g->canon[g->mip[l][v]];
    }
    free(g->canon); g->canon = NULL;
    table_free(&t);
    for (int64_t k = 0; k < nbins && bitrate; k++) {
        if (codebook) codebook[k] = ((double)(2 * k + 1)) / (double)(2 * nbins);
        if (sigma) sigma[k] = cnt[k] ? sqrt(ssq[k] / (double)cnt[k]) : 0.0;
    }
    free(ssq); free(cnt);
    if (n_picks) *n_picks = npick;
    return g;
}

/* The mixture a quantised graph reconstructs for one node: 1 pushed from the
 * node to the sources, q receiving the codeword of the node's bin (a) and p
 * the rest.  out: S doubles (dense). */
void mgo_quantised_mixture(const mgo_graph *g, const double *codebook, uint32_t node, double *out)
{
    size_t cap = 64, n = 0;
    uint32_t *sn = (uint32_t *)malloc(cap * sizeof(uint32_t));
    double *sw = (double *)malloc(cap * sizeof(double));
    sn[n] = node; sw[n] = 1.0; n++;
    while (n) {
        n--;
        uint32_t k = sn[n];
        double w = sw[n];
        if (k < g->S) { out[k] += w; continue; }
        double c = codebook[g->a[k]];
        if (n + 2 > cap) {
            cap *= 2;
            sn = (uint32_t *)realloc(sn, cap * sizeof(uint32_t));
            sw = (double *)realloc(sw, cap * sizeof(double));
        }
        sn[n] = g->p[k]; sw[n] = w * (1.0 - c); n++;
        sn[n] = g->q[k]; sw[n] = w * c; n++;
    }
    free(sn); free(sw);
}

/* The greedy factorisation of given mixtures (CSR lists ascending by ID,
 * integer weights), as mgo_build_greedy does for a volume's mipmap; roots[m]
 * receives the canonical node of mixture m.  For the paper's worked examples. */
mgo_graph *mgo_greedy_lists(const uint64_t *off, const uint32_t *ids, const uint64_t *cnt_in, int64_t M, uint32_t S,
                            int strategy, int tau, int bitrate, uint32_t *roots, uint32_t *picks, int64_t max_picks,
                            int64_t *n_picks)
{
    if ((strategy != 1 && strategy != 2) || bitrate < 0 || bitrate > 16 || tau < 1) return NULL;
    mgo_graph *g = (mgo_graph *)calloc(1, sizeof(mgo_graph));
    if (!g) return NULL;
    g->S = S;
    g->L = 0;
    gr_lists x;
    x.M = M;
    int64_t E = (int64_t)off[M];
    x.off = (int64_t *)malloc((size_t)(M + 1) * sizeof(int64_t));
    x.len = (int32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(int32_t));
    x.comp = (uint32_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(uint32_t));
    x.wt = (uint64_t *)malloc((size_t)(E > 0 ? E : 1) * sizeof(uint64_t));
    for (int64_t m = 0; m <= M; m++) x.off[m] = (int64_t)off[m];
    for (int64_t m = 0; m < M; m++) x.len[m] = (int32_t)(off[m + 1] - off[m]);
    for (int64_t e = 0; e < E; e++) { x.comp[e] = ids[e]; x.wt[e] = cnt_in[e]; }
    mgo_table t;
    table_init(&t, S);
    int64_t nbins = bitrate ? ((int64_t)1 << bitrate) : 1;
    double *ssq = (double *)calloc((size_t)nbins, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nbins, sizeof(int64_t));
    gr_run(&x, &t, strategy, tau, bitrate, ssq, cnt, picks, max_picks, n_picks);
    uint32_t *tmp = (uint32_t *)malloc((size_t)(M > 0 ? M : 1) * sizeof(uint32_t));
    for (int64_t m = 0; m < M; m++) tmp[m] = x.comp[x.off[m]];
    gr_free(&x);
    free(ssq); free(cnt);
    if (relabel(g, &t)) { free(tmp); table_free(&t); mgo_graph_free(g); return NULL; }
    for (int64_t m = 0; m < M; m++) roots[m] = (uint32_t)g->canon[tmp[m]];
    free(tmp);
    free(g->canon); g->canon = NULL;
    table_free(&t);
    return g;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.5 (Eq. 16-17) and Sec. 3.6: every node's mixture with its          */
/* uncertainty (the mixture lookup table), and box histograms summed from   */
/* it with error bars.                                                       */
/*                                                                          */
/* Readings taken here:                                                      */
/*   E1 node n's weight w_n is that of q (b/(a+b) exact, or the codeword of  */
/*      its bin), its uncertainty dw_n (0 exact, or the bin's sigma).        */
/*   E2 Eq. 17 per component i: mu_i(n) = (1 - w) mu_i(p) + w mu_i(q) and    */
/*      dmu_i(n)^2 = mu_i(n)^2 ((dmu_i(p)/mu_i(p))^2 + (dmu_i(q)/mu_i(q))^2  */
/*      + 2 (dw/w)^2), a ratio term being 0 when the component is absent     */
/*      from that input.  Sources: mu = e_s, dmu = 0.                        */
/*   E3 a box's histogram from the table: h_s = sum over its footprint       */
/*      cubes c (Algorithm 1) of W_c mu_s(node_c), W_c = 8^l; the error bar  */
/*      dh_s = sqrt(sum_c (W_c dmu_s(node_c))^2) (Eq. 16, independent sums). */
/* ------------------------------------------------------------------------ */
/* Rows of every node, sources ascending.  With src == NULL only off (N + 1)
 * is filled (sizes); returns 0, or -1 on a malformed table. */
int mgo_error_rows(const uint32_t *p, const uint32_t *q, const double *w, const double *dw, int64_t N, uint32_t S,
                   int64_t *off, uint32_t *src, double *mu, double *dmu)
{
    off[0] = 0;
    for (int64_t n = 0; n < N; n++) {
        if (n < S) { off[n + 1] = off[n] + 1; continue; }
        if (p[n] >= n || q[n] >= n) return -1;
        /* an upper bound (disjoint sources give exactly the sum) */
        off[n + 1] = off[n] + (off[p[n] + 1] - off[p[n]]) + (off[q[n] + 1] - off[q[n]]);
    }
    if (!src) return 0;
    for (int64_t n = 0; n < N; n++) {
        int64_t o = off[n];
        if (n < S) { src[o] = (uint32_t)n; mu[o] = 1.0; dmu[o] = 0.0; continue; }
        int64_t a = off[p[n]], ae = off[p[n] + 1], b = off[q[n]], be = off[q[n] + 1];
        double wq = w[n], wp = 1.0 - w[n];
        double rw = wq > 0 ? dw[n] / wq : 0.0;
        int64_t k = o;
        while (a < ae || b < be) {
            int from_a = b >= be || (a < ae && src[a] <= src[b]);
            int from_b = a >= ae || (b < be && src[b] <= src[a]);
            uint32_t s = from_a ? src[a] : src[b];
            double m = 0.0, r2 = 2.0 * rw * rw;
            if (from_a) { m += wp * mu[a]; if (mu[a] > 0) r2 += (dmu[a] / mu[a]) * (dmu[a] / mu[a]); a++; }
            if (from_b) { m += wq * mu[b]; if (mu[b] > 0) r2 += (dmu[b] / mu[b]) * (dmu[b] / mu[b]); b++; }
            src[k] = s; mu[k] = m; dmu[k] = sqrt(m * m * r2);
            k++;
        }
        for (; k < off[n + 1]; k++) { src[k] = 0xFFFFFFFFu; mu[k] = 0.0; dmu[k] = 0.0; }   /* unused slack */
    }
    return 0;
}

/* hist, err: Q x S (err may be NULL) */
void mgo_lut_query(const mgo_graph *g, const int64_t *off, const uint32_t *src, const double *mu, const double *dmu,
                   const int32_t *boxes, int64_t Q, double *hist, double *err)
{
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < Q; i++) {
        double *h = hist + i * (int64_t)g->S, *e = err ? err + i * (int64_t)g->S : NULL;
        for (uint32_t s = 0; s < g->S; s++) { h[s] = 0.0; if (e) e[s] = 0.0; }
        int64_t n = mgo_fa_cubes(boxes + 6 * i, nx, ny, nz, NULL, 0);
        if (n <= 0) continue;
        int32_t *cubes = (int32_t *)malloc((size_t)n * 4 * sizeof(int32_t));
        mgo_fa_cubes(boxes + 6 * i, nx, ny, nz, cubes, n);
        for (int64_t c = 0; c < n; c++) {
            int l = cubes[4 * c];
            const int64_t *d = g->dims + 3 * l;
            uint32_t node = g->mip[l][((int64_t)cubes[4 * c + 3] * d[1] + cubes[4 * c + 2]) * d[0] + cubes[4 * c + 1]];
            double W = ldexp(1.0, 3 * l);
            for (int64_t k = off[node]; k < off[node + 1]; k++) {
                if (src[k] == 0xFFFFFFFFu) continue;
                h[src[k]] += W * mu[k];
                if (e) e[src[k]] += (W * dmu[k]) * (W * dmu[k]);
            }
        }
        if (e) for (uint32_t s = 0; s < g->S; s++) e[s] = sqrt(e[s]);
        free(cubes);
    }
}
