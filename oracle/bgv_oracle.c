/*
 * bgv_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the BigGraphVis hot path
 * (Moradi & Mondal, "BigGraphVis: Leveraging Streaming Algorithms and GPU
 * Acceleration for Visualizing Big Graphs", arXiv 2108.00529).  It exists to
 * check the CUDA library; nothing in the product path may call it.  It shares
 * no code, header, table or constant generator with the CUDA sources.
 *
 * Integer stages (sketch, community passes, supergraph) are exact.  The
 * ForceAtlas2 stage computes forces in FP64; only the quantities that *decide*
 * the Barnes-Hut tree and its opening test are FP32, because those decisions
 * are taken in the kernel's precision on both sides (the tree frame, the
 * quantised body coordinates and the opening test).
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off matters: the FP32 decision arithmetic below must be
 * rounded operation by operation, never fused into FMAs.
 *
 * Readings of points the paper leaves open are stated where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EBADEDGE 3

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Hash family (Section 3.3: "pairwise independent hash functions").        */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): advance the state by the
 * golden-ratio increment and return the mixed value. */
uint64_t orc_splitmix64(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Reading (the paper names no hash): Carter-Wegman h_i(x) = ((a_i x + b_i)
 * mod p) mod w with p = 2^31 - 1.  Row i draws two SplitMix64 outputs from
 * state seed + i: a_i = 1 + z1 mod (p - 1), b_i = z2 mod p. */
void orc_hash_coeffs(uint64_t seed, int32_t rows, uint64_t *a, uint64_t *b)
{
    const uint64_t p = 2147483647ULL;
    for (int32_t i = 0; i < rows; ++i) {
        uint64_t st = seed + (uint64_t)i;
        uint64_t z1 = orc_splitmix64(&st);
        uint64_t z2 = orc_splitmix64(&st);
        a[i] = 1 + z1 % (p - 1);
        b[i] = z2 % p;
    }
}

uint32_t orc_hash(uint64_t a, uint64_t b, uint32_t x, uint32_t width)
{
    const uint64_t p = 2147483647ULL;
    return (uint32_t)(((a * (uint64_t)x + b) % p) % (uint64_t)width);
}

/* ------------------------------------------------------------------------ */
/* Degrees and the count-min sketch (Algorithm 2; Section 3.3).             */
/* ------------------------------------------------------------------------ */

static int check_edges(const int32_t *edges, int64_t m, int32_t n)
{
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || u >= n || v < 0 || v >= n) return ORC_EBADEDGE;
    }
    return ORC_OK;
}

/* Exact degrees: each endpoint of each edge counts once (a self-loop counts
 * twice for its node). */
int orc_exact_degrees(const int32_t *edges, int64_t m, int32_t n, uint32_t *deg)
{
    if (n < 0 || m < 0) return ORC_EINVAL;
    if (check_edges(edges, m, n)) return ORC_EBADEDGE;
    memset(deg, 0, sizeof(uint32_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        deg[edges[2 * e]] += 1;
        deg[edges[2 * e + 1]] += 1;
    }
    return ORC_OK;
}

/* Algorithm 2 taken literally: the events are the edge endpoints in stream
 * order; for every event x and every row i, M[i][h_i(x)] += 1.  The answer
 * for node v is min_i M[i][h_i(v)] (the "minimum value" of Algorithm 2,
 * Section 3.3).  S is rows x width, row-major. */
int orc_sketch_degrees(const int32_t *edges, int64_t m, int32_t n, int32_t rows, int32_t width,
                       uint64_t seed, uint32_t *S, uint32_t *dhat)
{
    uint64_t a[64], b[64];
    if (n < 0 || m < 0 || rows < 1 || rows > 64 || width < 1) return ORC_EINVAL;
    if (check_edges(edges, m, n)) return ORC_EBADEDGE;
    orc_hash_coeffs(seed, rows, a, b);
    memset(S, 0, sizeof(uint32_t) * (size_t)rows * (size_t)width);
    for (int64_t e = 0; e < m; ++e) {
        for (int k = 0; k < 2; ++k) {
            uint32_t x = (uint32_t)edges[2 * e + k];
            for (int32_t i = 0; i < rows; ++i)
                S[(size_t)i * width + orc_hash(a[i], b[i], x, (uint32_t)width)] += 1;
        }
    }
    for (int32_t v = 0; v < n; ++v) {
        uint32_t best = UINT32_MAX;
        for (int32_t i = 0; i < rows; ++i) {
            uint32_t c = S[(size_t)i * width + orc_hash(a[i], b[i], (uint32_t)v, (uint32_t)width)];
            if (c < best) best = c;
        }
        dhat[v] = best;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Community passes (Algorithm 3 rounds; Section 3.2.1; Section 4.2.2).      */
/* ------------------------------------------------------------------------ */

/* Reading of Algorithm 3 (synchronous, deterministic):
 *   c[v] = v, d[v] = dhat[v] (sketched degree), D = threshold.
 *   For each round: every edge (u, v), u != v, in edge-index order, reads the
 *   labels and degrees as they stood at the start of the round.  It is
 *   skipped unless d[u] <= D and d[v] <= D, and skipped when c[u] == c[v].
 *   If d[u] > d[v] it proposes that v take c[u]; if d[v] > d[u] that u take
 *   c[v]; on a tie it does nothing (tie_mode 0, the strict comparisons of
 *   Algorithm 3) or the lower id takes the higher id's label (tie_mode 1).
 *   At the end of the round every node with at least one proposal takes the
 *   proposal of the lowest edge index and its degree grows by one
 *   (saturating).  Then D = min(D * growth, 2^32 - 1) (Section 3.2.1: the
 *   threshold is multiplied by a constant factor each round). */
/* Mode degree (Section 4.2.2 "Community Detection": the most common degree
 * is the threshold SCoDA suggests): the most frequent value of dhat among
 * nodes with dhat >= 1; ties go to the smaller value; 0 when every dhat is
 * 0. */
static int cmp_u32(const void *x, const void *y)
{
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

int orc_mode_degree(const uint32_t *dhat, int32_t n, uint32_t *mode)
{
    if (n < 0 || !mode) return ORC_EINVAL;
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!v) return ORC_ENOMEM;
    int32_t k = 0;
    for (int32_t i = 0; i < n; ++i)
        if (dhat[i] >= 1) v[k++] = dhat[i];
    /* sort, then the longest run of equal values; runs are met in ascending
     * value order, so a strict improvement keeps the smaller value on ties */
    qsort(v, (size_t)k, sizeof(uint32_t), cmp_u32);
    uint32_t best = 0;
    int64_t best_count = 0;
    for (int32_t i = 0; i < k;) {
        int32_t j = i;
        while (j < k && v[j] == v[i]) ++j;
        if (j - i > best_count) {
            best = v[i];
            best_count = j - i;
        }
        i = j;
    }
    free(v);
    *mode = best;
    return ORC_OK;
}

/* Community passes (Algorithm 3 lines 8-22; Section 3.2.1).
 * Readings: degrees start at the sketched dhat and a node's degree grows by
 * one when it moves; both endpoints must be <= D; every edge reads the state
 * at the start of the pass, and a node with several proposals takes the one
 * of the lowest edge index; D <- min(D * growth, 2^32 - 1) after each pass,
 * with growth 0 meaning "multiply by the first-pass threshold", i.e. the
 * delta^i schedule of Section 4.2.2.  After each pass, `jumps` synchronous
 * pointer-jumping steps replace every label by its label's label. */
int orc_communities_ex(const int32_t *edges, int64_t m, int32_t n, const uint32_t *dhat, int32_t passes,
                       uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t jumps, int32_t *labels,
                       uint32_t *deg_out)
{
    if (n < 0 || m < 0 || passes < 0 || jumps < 0 || (tie_mode != 0 && tie_mode != 1)) return ORC_EINVAL;
    if (check_edges(edges, m, n)) return ORC_EBADEDGE;
    uint32_t *d = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *prop_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *prop_l = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!d || !prop_e || !prop_l) {
        free(d); free(prop_e); free(prop_l);
        return ORC_ENOMEM;
    }
    for (int32_t v = 0; v < n; ++v) {
        labels[v] = v;
        d[v] = dhat[v];
    }
    uint64_t D = threshold;
    const uint64_t factor = growth ? growth : threshold;
    for (int32_t p = 0; p < passes; ++p) {
        for (int32_t v = 0; v < n; ++v) prop_e[v] = -1;
        for (int64_t e = 0; e < m; ++e) {
            int32_t u = edges[2 * e], v = edges[2 * e + 1];
            int32_t join, lab;
            if (u == v) continue;
            if ((uint64_t)d[u] > D || (uint64_t)d[v] > D) continue;
            if (labels[u] == labels[v]) continue;
            if (d[u] > d[v]) {
                join = v; lab = labels[u];
            } else if (d[v] > d[u]) {
                join = u; lab = labels[v];
            } else if (tie_mode == 1) {
                join = u < v ? u : v;
                lab = labels[u < v ? v : u];
            } else {
                continue;
            }
            if (prop_e[join] < 0) {  /* first in edge order = lowest index */
                prop_e[join] = e;
                prop_l[join] = lab;
            }
        }
        for (int32_t v = 0; v < n; ++v) {
            if (prop_e[v] >= 0) {
                labels[v] = prop_l[v];
                if (d[v] != UINT32_MAX) d[v] += 1;
            }
        }
        for (int32_t j = 0; j < jumps; ++j) {
            for (int32_t v = 0; v < n; ++v) prop_l[v] = labels[labels[v]];
            memcpy(labels, prop_l, sizeof(int32_t) * (size_t)n);
        }
        D = D * factor;
        if (D > UINT32_MAX) D = UINT32_MAX;
    }
    if (deg_out) memcpy(deg_out, d, sizeof(uint32_t) * (size_t)n);
    free(d); free(prop_e); free(prop_l);
    return ORC_OK;
}

int orc_communities(const int32_t *edges, int64_t m, int32_t n, const uint32_t *dhat, int32_t passes,
                    uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t *labels,
                    uint32_t *deg_out)
{
    if (growth < 1) return ORC_EINVAL;
    return orc_communities_ex(edges, m, n, dhat, passes, threshold, growth, tie_mode, 0, labels, deg_out);
}

/* Sequential SCoDA (Hollocou et al. 2017, as Section 3.2 describes it): one
 * pass over the edges in order, every node starting at degree 0 in its own
 * community; each edge first increments both endpoint degrees, then, if
 * both are at most D, the endpoint of smaller degree joins the community of
 * the other (ties: the first endpoint joins the second's).  The prior art
 * the GPU rounds replace; used to compare community quality. */
int orc_scoda_sequential(const int32_t *edges, int64_t m, int32_t n, uint32_t D, int32_t *labels)
{
    if (n < 0 || m < 0) return ORC_EINVAL;
    if (check_edges(edges, m, n)) return ORC_EBADEDGE;
    uint32_t *d = (uint32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint32_t));
    if (!d) return ORC_ENOMEM;
    for (int32_t v = 0; v < n; ++v) labels[v] = v;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        if (u == v) continue;
        d[u] += 1;
        d[v] += 1;
        if (d[u] <= D && d[v] <= D) {
            if (d[u] > d[v]) labels[v] = labels[u];
            else labels[u] = labels[v];
        }
    }
    free(d);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Supergraph (Section 4.1; Algorithm 3 "Compute community sizes" and the    */
/* ForceAtlas2(Csrc, Cdst, Csize) call).                                     */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Supernodes are the distinct labels, numbered by ascending label
 * (node_map[v] = rank of labels[v]).  Superedges are the cut edges
 * (labels[u] != labels[v]) keyed (min(map u, map v), max(...)), sorted
 * ascending and collapsed into multiplicities w.  Community size (Section
 * 4.1): for each node v, M[i][h_i(labels[v])] += dhat[v]; the size of
 * community k is min_i M[i][h_i(label_k)].  Reading: mass[k] = 1 + that size,
 * saturated to 2^32 - 1, so isolated communities keep a positive mass.  The
 * symmetric CSR lists, for each supernode, its neighbours in ascending order
 * with the superedge weight.  vol[k] (exact sum of dhat) and count[k] (nodes)
 * are diagnostics.  Output arrays may be NULL where marked optional. */
int orc_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels,
                   const uint32_t *dhat, int32_t rows, int32_t width, uint64_t seed,
                   int32_t *node_map, int64_t *K_out, int32_t *ssrc, int32_t *sdst, uint32_t *sw,
                   int64_t *Es_out, uint32_t *mass, uint64_t *vol /*opt*/, uint32_t *count /*opt*/,
                   int32_t *comm_label /*opt*/, int32_t *csr_off /*opt*/, int32_t *csr_adj /*opt*/,
                   uint32_t *csr_w /*opt*/)
{
    uint64_t a[64], b[64];
    if (n < 0 || m < 0 || rows < 1 || rows > 64 || width < 1) return ORC_EINVAL;
    if (check_edges(edges, m, n)) return ORC_EBADEDGE;
    for (int32_t v = 0; v < n; ++v)
        if (labels[v] < 0 || labels[v] >= n) return ORC_EINVAL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *label_of = (int32_t *)malloc(sizeof(int32_t) * nn);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
    uint64_t *M = (uint64_t *)calloc((size_t)rows * (size_t)width, sizeof(uint64_t));
    if (!rank || !label_of || !keys || !M) {
        free(rank); free(label_of); free(keys); free(M);
        return ORC_ENOMEM;
    }
    /* distinct labels in ascending order */
    for (int32_t l = 0; l < n; ++l) rank[l] = -1;
    for (int32_t v = 0; v < n; ++v) rank[labels[v]] = 0;
    int64_t K = 0;
    for (int32_t l = 0; l < n; ++l)
        if (rank[l] == 0) {
            rank[l] = (int32_t)K;
            label_of[K] = l;
            ++K;
        }
    for (int32_t v = 0; v < n; ++v) node_map[v] = rank[labels[v]];
    /* cut-edge keys */
    int64_t mc = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        if (labels[u] == labels[v]) continue;
        uint64_t x = (uint64_t)node_map[u], y = (uint64_t)node_map[v];
        uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
        keys[mc++] = (lo << 32) | hi;
    }
    qsort(keys, (size_t)mc, sizeof(uint64_t), cmp_u64);
    int64_t Es = 0;
    for (int64_t i = 0; i < mc; ++i) {
        if (i == 0 || keys[i] != keys[i - 1]) {
            ssrc[Es] = (int32_t)(keys[i] >> 32);
            sdst[Es] = (int32_t)(keys[i] & 0xFFFFFFFFULL);
            sw[Es] = 1;
            ++Es;
        } else {
            sw[Es - 1] += 1;
        }
    }
    /* community-size sketch */
    orc_hash_coeffs(seed, rows, a, b);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t i = 0; i < rows; ++i)
            M[(size_t)i * width + orc_hash(a[i], b[i], (uint32_t)labels[v], (uint32_t)width)] += dhat[v];
    for (int64_t k = 0; k < K; ++k) {
        uint64_t best = UINT64_MAX;
        for (int32_t i = 0; i < rows; ++i) {
            uint64_t c = M[(size_t)i * width + orc_hash(a[i], b[i], (uint32_t)label_of[k], (uint32_t)width)];
            if (c < best) best = c;
        }
        uint64_t ms = best + 1;
        mass[k] = ms > UINT32_MAX ? UINT32_MAX : (uint32_t)ms;
        if (comm_label) comm_label[k] = label_of[k];
    }
    if (vol) {
        memset(vol, 0, sizeof(uint64_t) * (size_t)(K > 0 ? K : 1));
        for (int32_t v = 0; v < n; ++v) vol[node_map[v]] += dhat[v];
    }
    if (count) {
        memset(count, 0, sizeof(uint32_t) * (size_t)(K > 0 ? K : 1));
        for (int32_t v = 0; v < n; ++v) count[node_map[v]] += 1;
    }
    /* symmetric CSR: both directions of every superedge, sorted by (row, col) */
    if (csr_off && csr_adj && csr_w) {
        uint64_t *dir = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * Es > 0 ? 2 * Es : 1));
        if (!dir) {
            free(rank); free(label_of); free(keys); free(M);
            return ORC_ENOMEM;
        }
        for (int64_t s = 0; s < Es; ++s) {
            dir[2 * s] = ((uint64_t)ssrc[s] << 32) | (uint64_t)sdst[s];
            dir[2 * s + 1] = ((uint64_t)sdst[s] << 32) | (uint64_t)ssrc[s];
        }
        qsort(dir, (size_t)(2 * Es), sizeof(uint64_t), cmp_u64);
        for (int64_t k = 0; k <= K; ++k) csr_off[k] = 0;
        for (int64_t t = 0; t < 2 * Es; ++t) csr_off[(dir[t] >> 32) + 1] += 1;
        for (int64_t k = 0; k < K; ++k) csr_off[k + 1] += csr_off[k];
        for (int64_t t = 0; t < 2 * Es; ++t) {
            int32_t r = (int32_t)(dir[t] >> 32), c = (int32_t)(dir[t] & 0xFFFFFFFFULL);
            csr_adj[t] = c;
            /* weight of the undirected superedge (min, max): binary search */
            int32_t lo = r < c ? r : c, hi = r < c ? c : r;
            uint64_t key = ((uint64_t)lo << 32) | (uint64_t)hi;
            int64_t L = 0, R = Es;
            while (L < R) {
                int64_t mid = (L + R) / 2;
                uint64_t km = ((uint64_t)ssrc[mid] << 32) | (uint64_t)sdst[mid];
                if (km < key) L = mid + 1; else R = mid;
            }
            csr_w[t] = sw[L];
        }
        free(dir);
    }
    *K_out = K;
    *Es_out = Es;
    free(rank); free(label_of); free(keys); free(M);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Modularity (the equation of Section "Quantity measure").                   */
/* ------------------------------------------------------------------------ */

/* Q = 1/(2m) sum_ij [A_ij - k_i k_j / (2m)] [C_i == C_j] for a simple
 * undirected graph, evaluated per community as sum_c (2 e_c)/(2m) -
 * (vol_c / 2m)^2 where e_c counts the edges inside c and vol_c sums degrees. */
double orc_modularity(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels)
{
    if (m <= 0 || n <= 0) return 0.0;
    double *in = (double *)calloc((size_t)n, sizeof(double));
    double *vol = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        vol[labels[u]] += 1.0;
        vol[labels[v]] += 1.0;
        if (labels[u] == labels[v]) in[labels[u]] += 2.0;
    }
    double two_m = 2.0 * (double)m, q = 0.0;
    for (int32_t c = 0; c < n; ++c) q += in[c] / two_m - (vol[c] / two_m) * (vol[c] / two_m);
    free(in); free(vol);
    return q;
}

/* ------------------------------------------------------------------------ */
/* ForceAtlas2 (Section 3.1, Algorithm 1; model of Jacomy et al. 2014).       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double theta;   /* Barnes-Hut opening parameter */
    double kr;      /* repulsion scaling */
    double kg;      /* gravity */
    double tau;     /* jitter tolerance */
    double ks;      /* local speed constant */
    double ksmax;   /* local speed cap constant */
    int32_t strong_gravity;
    int32_t leaf_cap;
    int32_t max_depth; /* L: levels of the quadtree, 1..24 */
    int32_t reserved;
} orc_fa2_params;

/* Initial positions (Algorithm 1: "Pos_i = random(space)").  Reading: the
 * space is the square [-sqrt K, sqrt K)^2; coordinate `axis` of node i uses
 * the SplitMix64 output for state seed + 2 i + axis, its top 24 bits as a
 * uniform U in [0, 1), and p = U * (2 R) - R with R = sqrt(K), all in FP32. */
void orc_fa2_init(int64_t K, uint64_t seed, float *pos)
{
    float R = sqrtf((float)K);
    float R2 = R * 2.0f;
    for (int64_t i = 0; i < K; ++i) {
        for (int axis = 0; axis < 2; ++axis) {
            uint64_t st = seed + 2 * (uint64_t)i + (uint64_t)axis;
            uint64_t z = orc_splitmix64(&st);
            float U = (float)(z >> 40) * 0x1p-24f;
            float t = U * R2;
            pos[2 * i + axis] = t - R;
        }
    }
}

/* ---- the quadtree that both sides build --------------------------------
 * Frame: lo = min over bodies of the FP32 coordinates; ext = max(hi.x - lo.x,
 * hi.y - lo.y); side = ext * (1 + 2^-20) (side = 1 when ext is 0).  All FP32.
 * Fixed-point body coordinate: U = trunc(((p - lo) / side) * 2^32) in FP32
 * arithmetic, so 0 <= U < 2^32.  Quantised coordinate q = U >> (32 - L).
 * Digit at level l (0 = top) = 2 * bit(qx, L-1-l) + bit(qy, L-1-l).
 * A cell is a digit prefix holding at least one body; it is split while it
 * holds more than leaf_cap bodies and its level is below L.
 * Opening test for body i and a non-leaf cell not containing i, all FP32:
 *   decision centre c = lo + side * (float(floor(SumU / M)) * 2^-32) per axis,
 *   where M = sum of body masses and SumU = sum of mass * U over the cell
 *   (exact integers, so the centre does not depend on summation order);
 *   dx = x_i - c.x, dy = y_i - c.y, d2 = dx*dx + dy*dy;
 *   accept iff s*s < (theta*theta) * d2 with s = side * 2^-level.
 * An accepted cell contributes with its FP64 centre of mass; a leaf is
 * summed body by body (excluding i); a cell containing i is always opened. */

typedef struct {
    int32_t level;
    int32_t is_leaf;
    int64_t start, end;  /* bodies [start, end) in key order */
    int32_t child[4];
    uint64_t M;
    u128 SX, SY;
    double cx, cy;      /* FP64 centre of mass */
    float dcx, dcy;     /* decision centre (FP32) */
    float side2;        /* (side * 2^-level)^2, FP32 */
} ocell;

typedef struct {
    int64_t K;
    int32_t L, leaf_cap;
    float lox, loy, side;
    uint64_t *key;      /* by body */
    uint32_t *Ux, *Uy;  /* by body */
    int64_t *order;     /* key order -> body */
    int64_t *pos_of;    /* body -> position in key order */
    ocell *cells;
    int64_t ncells, cap;
    const uint32_t *mass;
    const double *pos;
} otree;

static otree *g_sort_tree;
static int cmp_body(const void *x, const void *y)
{
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    uint64_t ki = g_sort_tree->key[i], kj = g_sort_tree->key[j];
    if (ki != kj) return ki < kj ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

static int digit_at(const otree *t, uint64_t key, int32_t level)
{
    return (int)((key >> (2 * (t->L - 1 - level))) & 3ULL);
}

static int32_t tree_build(otree *t, int32_t level, int64_t start, int64_t end)
{
    if (t->ncells == t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 1024;
        ocell *p = (ocell *)realloc(t->cells, sizeof(ocell) * (size_t)nc);
        if (!p) return -1;
        t->cells = p;
        t->cap = nc;
    }
    int32_t id = (int32_t)t->ncells++;
    ocell c;
    memset(&c, 0, sizeof(c));
    c.level = level;
    c.start = start;
    c.end = end;
    for (int q = 0; q < 4; ++q) c.child[q] = -1;
    double sx = 0.0, sy = 0.0;
    for (int64_t s = start; s < end; ++s) {
        int64_t i = t->order[s];
        uint64_t mi = t->mass[i];
        c.M += mi;
        c.SX += (u128)mi * (u128)t->Ux[i];
        c.SY += (u128)mi * (u128)t->Uy[i];
        sx += (double)mi * t->pos[2 * i];
        sy += (double)mi * t->pos[2 * i + 1];
    }
    c.cx = sx / (double)c.M;
    c.cy = sy / (double)c.M;
    {
        uint32_t qx = c.M ? (uint32_t)(c.SX / (u128)c.M) : 0u;
        uint32_t qy = c.M ? (uint32_t)(c.SY / (u128)c.M) : 0u;
        float fx = (float)qx;
        float fy = (float)qy;
        float ux = fx * 0x1p-32f;
        float uy = fy * 0x1p-32f;
        float ox = t->side * ux;
        float oy = t->side * uy;
        c.dcx = t->lox + ox;
        c.dcy = t->loy + oy;
        float s = ldexpf(t->side, -level);
        c.side2 = s * s;
    }
    c.is_leaf = (end - start <= t->leaf_cap) || level == t->L;
    t->cells[id] = c;
    if (!c.is_leaf) {
        int64_t s = start;
        for (int q = 0; q < 4; ++q) {
            int64_t e = s;
            while (e < end && digit_at(t, t->key[t->order[e]], level) == q) ++e;
            if (e > s) {
                int32_t ch = tree_build(t, level + 1, s, e);
                if (ch < 0) return -1;
                t->cells[id].child[q] = ch;
            }
            s = e;
        }
    }
    return id;
}

static void tree_free(otree *t)
{
    free(t->key); free(t->Ux); free(t->Uy); free(t->order); free(t->pos_of); free(t->cells);
    memset(t, 0, sizeof(*t));
}

/* Frame, keys, key order and the literal quadtree for K >= 1 bodies. */
static int tree_make(otree *t, int64_t K, const double *pos, const uint32_t *mass, int32_t leaf_cap, int32_t L)
{
    memset(t, 0, sizeof(*t));
    if (K < 1 || L < 1 || L > 24 || leaf_cap < 1) return ORC_EINVAL;
    t->K = K; t->L = L; t->leaf_cap = leaf_cap; t->mass = mass; t->pos = pos;
    float lx = (float)pos[0], ly = (float)pos[1], hx = lx, hy = ly;
    for (int64_t i = 1; i < K; ++i) {
        float x = (float)pos[2 * i], y = (float)pos[2 * i + 1];
        if (x < lx) lx = x;
        if (x > hx) hx = x;
        if (y < ly) ly = y;
        if (y > hy) hy = y;
    }
    float ex = hx - lx, ey = hy - ly;
    float ext = ex > ey ? ex : ey;
    float side = ext * (1.0f + 0x1p-20f);
    if (!(ext > 0.0f)) side = 1.0f;
    t->lox = lx; t->loy = ly; t->side = side;
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)K);
    t->Ux = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)K);
    t->Uy = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)K);
    t->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    t->pos_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (!t->key || !t->Ux || !t->Uy || !t->order || !t->pos_of) {
        tree_free(t);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < K; ++i) {
        float x = (float)pos[2 * i], y = (float)pos[2 * i + 1];
        float dx = x - lx, dy = y - ly;
        float ux = dx / side, uy = dy / side;
        float sx = ux * 4294967296.0f, sy = uy * 4294967296.0f;
        uint32_t Ux = (uint32_t)sx, Uy = (uint32_t)sy;
        uint32_t qx = Ux >> (32 - L), qy = Uy >> (32 - L);
        uint64_t key = 0;
        for (int32_t l = 0; l < L; ++l) {
            uint64_t d = (uint64_t)((((qx >> (L - 1 - l)) & 1u) << 1) | ((qy >> (L - 1 - l)) & 1u));
            key = (key << 2) | d;
        }
        t->Ux[i] = Ux; t->Uy[i] = Uy; t->key[i] = key; t->order[i] = i;
    }
    g_sort_tree = t;
    qsort(t->order, (size_t)K, sizeof(int64_t), cmp_body);
    for (int64_t s = 0; s < K; ++s) t->pos_of[t->order[s]] = s;
    if (tree_build(t, 0, 0, K) < 0) {
        tree_free(t);
        return ORC_ENOMEM;
    }
    return ORC_OK;
}

typedef struct {
    const otree *t;
    int64_t i, si;      /* body and its key-order position */
    double xi, yi, mi;  /* FP64 */
    float fxi, fyi;     /* FP32 copies for the opening test */
    float theta2;
    double kr;
    double fx, fy;
    int64_t inter;
} ovisit;

static void add_point(ovisit *v, double px, double py, double pm)
{
    double dx = v->xi - px, dy = v->yi - py;
    double d2 = dx * dx + dy * dy;
    v->inter += 1;
    if (d2 > 0.0) {
        double f = v->kr * v->mi * pm / d2;
        v->fx += f * dx;
        v->fy += f * dy;
    }
}

static void visit_cell(ovisit *v, int32_t id)
{
    const otree *t = v->t;
    const ocell *c = &t->cells[id];
    if (c->is_leaf) {
        for (int64_t s = c->start; s < c->end; ++s) {
            int64_t j = t->order[s];
            if (j == v->i) continue;
            add_point(v, t->pos[2 * j], t->pos[2 * j + 1], (double)t->mass[j]);
        }
        return;
    }
    int own = v->si >= c->start && v->si < c->end;
    if (!own) {
        float dx = v->fxi - c->dcx;
        float dy = v->fyi - c->dcy;
        float ax = dx * dx;
        float ay = dy * dy;
        float d2 = ax + ay;
        float rhs = v->theta2 * d2;
        if (c->side2 < rhs) {
            add_point(v, c->cx, c->cy, (double)c->M);
            return;
        }
    }
    for (int q = 0; q < 4; ++q)
        if (c->child[q] >= 0) visit_cell(v, c->child[q]);
}

/* Barnes-Hut repulsion (Section 3.1 "Body Repulsion"; node weights as masses,
 * Section 5.1): F_i = sum over accepted cells and leaf bodies j != i of
 * kr * m_i * m_j * (p_i - p_j) / |p_i - p_j|^2, zero for coincident points.
 * `which` (optional) restricts the output to listed bodies; Fr then holds
 * 2*count values in list order.  *interactions counts body-cell and
 * body-body terms. */
int orc_bh_repulsion(int64_t K, const double *pos, const uint32_t *mass, const orc_fa2_params *p,
                     const int64_t *which, int64_t count, double *Fr, int64_t *interactions)
{
    otree t;
    int64_t total = 0;
    if (K < 0) return ORC_EINVAL;
    int64_t nout = which ? count : K;
    if (K == 0) {
        if (interactions) *interactions = 0;
        return ORC_OK;
    }
    int rc = tree_make(&t, K, pos, mass, p->leaf_cap, p->max_depth);
    if (rc) return rc;
    float th = (float)p->theta;
    for (int64_t r = 0; r < nout; ++r) {
        int64_t i = which ? which[r] : r;
        ovisit v;
        memset(&v, 0, sizeof(v));
        v.t = &t; v.i = i; v.si = t.pos_of[i];
        v.xi = pos[2 * i]; v.yi = pos[2 * i + 1]; v.mi = (double)mass[i];
        v.fxi = (float)pos[2 * i]; v.fyi = (float)pos[2 * i + 1];
        v.theta2 = th * th;
        v.kr = p->kr;
        visit_cell(&v, 0);
        Fr[2 * r] = v.fx;
        Fr[2 * r + 1] = v.fy;
        total += v.inter;
    }
    if (interactions) *interactions = total;
    tree_free(&t);
    return ORC_OK;
}

/* Export the literal quadtree for structural checks.  Arrays sized max_cells;
 * returns the cell count (or -1 when max_cells is too small, -2 on error).
 * order[K] receives the key order (body ids). */
int64_t orc_quadtree_export(int64_t K, const double *pos, const uint32_t *mass, int32_t leaf_cap, int32_t L,
                            int64_t max_cells, int32_t *level, int32_t *is_leaf, int64_t *start, int64_t *end,
                            int32_t *child /*[4*max]*/, uint64_t *cmass, double *com /*[2*max]*/,
                            float *dcom /*[2*max]*/, int64_t *order, float *frame /*[3]*/)
{
    otree t;
    if (tree_make(&t, K, pos, mass, leaf_cap, L)) return -2;
    if (t.ncells > max_cells) {
        tree_free(&t);
        return -1;
    }
    for (int64_t c = 0; c < t.ncells; ++c) {
        level[c] = t.cells[c].level;
        is_leaf[c] = t.cells[c].is_leaf;
        start[c] = t.cells[c].start;
        end[c] = t.cells[c].end;
        for (int q = 0; q < 4; ++q) child[4 * c + q] = t.cells[c].child[q];
        cmass[c] = t.cells[c].M;
        com[2 * c] = t.cells[c].cx;
        com[2 * c + 1] = t.cells[c].cy;
        dcom[2 * c] = t.cells[c].dcx;
        dcom[2 * c + 1] = t.cells[c].dcy;
    }
    for (int64_t s = 0; s < K; ++s) order[s] = t.order[s];
    frame[0] = t.lox; frame[1] = t.loy; frame[2] = t.side;
    int64_t nc = t.ncells;
    tree_free(&t);
    return nc;
}

/* Exact all-pairs repulsion in FP64 (no tree). */
int orc_exact_repulsion(int64_t K, const double *pos, const uint32_t *mass, double kr, double *Fr)
{
    for (int64_t i = 0; i < K; ++i) {
        double fx = 0.0, fy = 0.0;
        for (int64_t j = 0; j < K; ++j) {
            if (j == i) continue;
            double dx = pos[2 * i] - pos[2 * j], dy = pos[2 * i + 1] - pos[2 * j + 1];
            double d2 = dx * dx + dy * dy;
            if (d2 > 0.0) {
                double f = kr * (double)mass[i] * (double)mass[j] / d2;
                fx += f * dx;
                fy += f * dy;
            }
        }
        Fr[2 * i] = fx;
        Fr[2 * i + 1] = fy;
    }
    return ORC_OK;
}

/* Linear attraction along weighted edges (Section 3.1 "Attractive Force";
 * FA2's linear model with edge-weight influence 1):
 * F_i = - sum over CSR neighbours j of w_ij * (p_i - p_j). */
int orc_attraction(int64_t K, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                   const double *pos, double *Fa)
{
    for (int64_t i = 0; i < K; ++i) {
        double fx = 0.0, fy = 0.0;
        for (int32_t t = csr_off[i]; t < csr_off[i + 1]; ++t) {
            int32_t j = csr_adj[t];
            double w = (double)csr_w[t];
            fx -= w * (pos[2 * i] - pos[2 * j]);
            fy -= w * (pos[2 * i + 1] - pos[2 * j + 1]);
        }
        Fa[2 * i] = fx;
        Fa[2 * i + 1] = fy;
    }
    return ORC_OK;
}

/* Gravity (Section 3.1 "Gravity"; Algorithm 1 "FM_i <- FM_i - Pos_i"):
 * F_i = -kg * m_i * p_i / |p_i| (zero at the origin); strong gravity:
 * F_i = -kg * m_i * p_i. */
int orc_gravity(int64_t K, const uint32_t *mass, const double *pos, double kg, int32_t strong, double *Fg)
{
    for (int64_t i = 0; i < K; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1], m = (double)mass[i];
        double r = sqrt(x * x + y * y);
        if (strong) {
            Fg[2 * i] = -kg * m * x;
            Fg[2 * i + 1] = -kg * m * y;
        } else if (r > 0.0) {
            Fg[2 * i] = -kg * m * x / r;
            Fg[2 * i + 1] = -kg * m * y / r;
        } else {
            Fg[2 * i] = 0.0;
            Fg[2 * i + 1] = 0.0;
        }
    }
    return ORC_OK;
}

/* One ForceAtlas2 iteration (Algorithm 1, body of the iteration loop; the
 * adaptive speed of Jacomy et al. 2014, Section "Adaptive speed"):
 *   F = repulsion + attraction + gravity;
 *   swing_i = |F_i - Fprev_i|, traction_i = |F_i + Fprev_i| / 2;
 *   S = sum m_i swing_i, T = sum m_i traction_i;
 *   if S > 0: speed += min(tau * T / S - speed, 0.5 * speed);
 *   s_i = ks * speed / (1 + speed * sqrt(swing_i)), capped at ksmax / |F_i|;
 *   p_i += s_i F_i; Fprev = F.
 * pos, Fprev and *speed are updated in place (FP64 state).  Optional
 * outputs: F (2K), ST[2] = {S, T}, *interactions. */
int orc_fa2_step(int64_t K, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                 const uint32_t *mass, const orc_fa2_params *p, double *pos, double *Fprev, double *speed,
                 double *F_out, double *ST, int64_t *interactions)
{
    if (K < 0) return ORC_EINVAL;
    size_t kk = (size_t)(K > 0 ? K : 1);
    double *Fr = (double *)malloc(sizeof(double) * 2 * kk);
    double *Fa = (double *)malloc(sizeof(double) * 2 * kk);
    double *Fg = (double *)malloc(sizeof(double) * 2 * kk);
    if (!Fr || !Fa || !Fg) {
        free(Fr); free(Fa); free(Fg);
        return ORC_ENOMEM;
    }
    int rc = orc_bh_repulsion(K, pos, mass, p, NULL, 0, Fr, interactions);
    if (rc) {
        free(Fr); free(Fa); free(Fg);
        return rc;
    }
    orc_attraction(K, csr_off, csr_adj, csr_w, pos, Fa);
    orc_gravity(K, mass, pos, p->kg, p->strong_gravity, Fg);
    double S = 0.0, T = 0.0;
    for (int64_t i = 0; i < K; ++i) {
        for (int a = 0; a < 2; ++a) Fr[2 * i + a] = Fr[2 * i + a] + Fa[2 * i + a] + Fg[2 * i + a];
        double sx = Fr[2 * i] - Fprev[2 * i], sy = Fr[2 * i + 1] - Fprev[2 * i + 1];
        double tx = Fr[2 * i] + Fprev[2 * i], ty = Fr[2 * i + 1] + Fprev[2 * i + 1];
        S += (double)mass[i] * sqrt(sx * sx + sy * sy);
        T += (double)mass[i] * sqrt(tx * tx + ty * ty) / 2.0;
    }
    if (S > 0.0) {
        double target = p->tau * T / S;
        double rise = target - *speed;
        double cap = 0.5 * *speed;
        *speed += rise < cap ? rise : cap;
    }
    for (int64_t i = 0; i < K; ++i) {
        double fx = Fr[2 * i], fy = Fr[2 * i + 1];
        double sx = fx - Fprev[2 * i], sy = fy - Fprev[2 * i + 1];
        double swing = sqrt(sx * sx + sy * sy);
        double fn = sqrt(fx * fx + fy * fy);
        double s = p->ks * *speed / (1.0 + *speed * sqrt(swing));
        if (fn > 0.0 && s * fn > p->ksmax) s = p->ksmax / fn;
        pos[2 * i] += s * fx;
        pos[2 * i + 1] += s * fy;
        Fprev[2 * i] = fx;
        Fprev[2 * i + 1] = fy;
        if (F_out) {
            F_out[2 * i] = fx;
            F_out[2 * i + 1] = fy;
        }
    }
    if (ST) {
        ST[0] = S;
        ST[1] = T;
    }
    free(Fr); free(Fa); free(Fg);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Supernode colours (Section 4.3).                                           */
/* ------------------------------------------------------------------------ */

static const uint32_t *g_sizes;
static int cmp_by_size(const void *x, const void *y)
{
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    if (g_sizes[i] != g_sizes[j]) return g_sizes[i] < g_sizes[j] ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

/* Section 4.3: with alpha the sum of all community sizes, the smallest
 * communities that together take half of alpha are drawn brown (group 0);
 * the rest are split into ten groups from small to big (groups 1..10).
 * Reading: order by size ascending (ties by id); group 0 holds the longest
 * prefix whose sizes sum to at most alpha / 2; the remaining R communities,
 * in the same order, get group 1 + floor(10 * rank / R). */
int orc_colour_groups(int64_t K, const uint32_t *size, uint8_t *group)
{
    if (K < 0) return ORC_EINVAL;
    if (K == 0) return ORC_OK;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (!order) return ORC_ENOMEM;
    uint64_t total = 0;
    for (int64_t k = 0; k < K; ++k) {
        order[k] = k;
        total += size[k];
    }
    g_sizes = size;
    qsort(order, (size_t)K, sizeof(int64_t), cmp_by_size);
    uint64_t cum = 0;
    int64_t half = 0;
    while (half < K && 2 * (cum + size[order[half]]) <= total) {
        cum += size[order[half]];
        ++half;
    }
    int64_t rest = K - half;
    for (int64_t r = 0; r < K; ++r) {
        int64_t k = order[r];
        if (r < half) group[k] = 0;
        else group[k] = (uint8_t)(1 + (10 * (r - half)) / rest);
    }
    free(order);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Drawing the supergraph (Section 4.1: radius proportional to the square   */
/* root of the size; Section 4.3: eleven colour groups) into an RGBA image.  */
/* ------------------------------------------------------------------------ */

/* Reading: the image maps the discs' bounding box [min(x - r), max(x + r)]
 * to the W x H pixels with one scale s = min(W, H) / (largest extent) (1 if
 * the extent is 0), origin at the box's low corner.  Pixel (px, py) shows
 * the disc whose centre (u, v) = ((x - lo_x) s, (y - lo_y) s) and radius
 * r s cover its centre (px + 0.5, py + 0.5): (px + 0.5 - u)^2 + (py + 0.5 -
 * v)^2 <= (r s)^2.  Where discs overlap the smaller radius is drawn on top,
 * equal radii by the smaller id, so small communities stay visible.  All in
 * FP32, operation by operation.  Colours: group 0 brown, groups 1..10 light
 * purple, purple, light orange, orange, light red, red, light green, green,
 * light blue, blue (the ColorBrewer "Paired" qualitative scheme); background
 * white; alpha 255.  Pixel-centric brute force over all discs. */
static const uint8_t orc_palette[11][3] = {
    {177, 89, 40},   {202, 178, 214}, {106, 61, 154}, {253, 191, 111}, {255, 127, 0}, {251, 154, 153},
    {227, 26, 28},   {178, 223, 138}, {51, 160, 44},  {166, 206, 227}, {31, 120, 180}};

int orc_render(int64_t K, const float *xy, const float *radius, const uint8_t *group, int32_t W, int32_t H,
               uint8_t *rgba)
{
    if (K < 0 || W < 1 || H < 1) return ORC_EINVAL;
    float lx = INFINITY, ly = INFINITY, hx = -INFINITY, hy = -INFINITY;
    for (int64_t k = 0; k < K; ++k) {
        float x = xy[2 * k], y = xy[2 * k + 1], r = radius[k];
        float a = x - r, b = y - r, c = x + r, d = y + r;
        if (a < lx) lx = a;
        if (b < ly) ly = b;
        if (c > hx) hx = c;
        if (d > hy) hy = d;
    }
    float ex = hx - lx, ey = hy - ly;
    float ext = ex > ey ? ex : ey;
    float s = (K > 0 && ext > 0.0f) ? (float)(W < H ? W : H) / ext : 1.0f;
    for (int32_t py = 0; py < H; ++py) {
        for (int32_t px = 0; px < W; ++px) {
            int64_t best = -1;
            float best_r = 0.0f;
            float cx = (float)px + 0.5f, cy = (float)py + 0.5f;
            for (int64_t k = 0; k < K; ++k) {
                float u = (xy[2 * k] - lx) * s, v = (xy[2 * k + 1] - ly) * s, rs = radius[k] * s;
                float dx = cx - u, dy = cy - v;
                float d2 = dx * dx + dy * dy;
                if (d2 <= rs * rs) {
                    if (best < 0 || radius[k] < best_r) {  /* k ascends, so ties keep the smaller id */
                        best = k;
                        best_r = radius[k];
                    }
                }
            }
            uint8_t *o = rgba + 4 * ((size_t)py * (size_t)W + (size_t)px);
            if (best < 0) {
                o[0] = o[1] = o[2] = 255;
            } else {
                const uint8_t *c = orc_palette[group[best] <= 10 ? group[best] : 0];
                o[0] = c[0]; o[1] = c[1]; o[2] = c[2];
            }
            o[3] = 255;
        }
    }
    return ORC_OK;
}
