/*
 * bgv.h -- C ABI of the GB300 BigGraphVis hot-path library (libbgv.so).
 *
 * The method: Moradi & Mondal, "BigGraphVis: Leveraging Streaming Algorithms
 * and GPU Acceleration for Visualizing Big Graphs" (arXiv 2108.00529).  The
 * library computes, on one GPU,
 *   1. a count-min sketch of node degrees (Algorithm 2, Section 3.3),
 *   2. streaming community labels over a few rounds on the edge list
 *      (Algorithm 3, Section 3.2.1),
 *   3. the supergraph: communities as supernodes with sketched sizes as
 *      masses, cut edges merged into weighted superedges (Section 4.1),
 *   4. ForceAtlas2 iterations on that supergraph (Section 3.1, Algorithm 1):
 *      Barnes-Hut repulsion on a quadtree, attraction along weighted edges,
 *      gravity, per-node swing and an adaptive global speed.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.   Array arguments are DEVICE pointers owned by the caller, unless
 *             the entry point's name ends in _host.  The library never keeps a
 *             pointer after the call's work on `stream` has finished.
 * Streams.    `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *             default stream).  Calls only enqueue work; they do not
 *             synchronise, except bgv_status, bgv_fa2_read_stats and the
 *             bgv_layout* pipeline calls (documented there).  A ForceAtlas2
 *             step forks its work from `stream` onto two library streams of
 *             the calling host thread and device (the main chain at the
 *             device's highest stream priority, the attraction beside it)
 *             and joins them back into `stream` before it returns, so its
 *             work is ordered on `stream` like any other call.  Those
 *             streams are made by the first such call of a host thread on a
 *             device (make it outside any stream capture) and live until the
 *             process ends; each step makes and destroys four CUDA events.
 * Scratch.    The library allocates no memory.  Each stage takes a caller
 *             workspace `ws` of `ws_bytes` bytes (256-byte aligned), sized by
 *             the matching *_ws_size query.  The first 256 bytes of every
 *             workspace hold a status word and counters; the rest is scratch
 *             whose contents do not outlive the call, except where stated
 *             (bgv_fa2_step keeps per-step statistics there).
 * Status.     Every call returns an int: BGV_OK, or an error detected on the
 *             host before any work is enqueued (BGV_EINVAL, BGV_ENOSPC), or
 *             BGV_ECUDA when a launch fails.  Errors found on the device (an
 *             edge endpoint outside [0, n), a label outside [0, n), a bounded
 *             wait that gave up) are OR-ed into the status word in the
 *             workspace as BGV_DEV_* bits; read them with bgv_status.
 *             Outputs of a call whose status word is non-zero are undefined.
 * Sizes.      Data-dependent sizes (K communities, Es superedges) are written
 *             to device int64 scalars, so a chain of calls needs no host
 *             round trip.  Callers size outputs by their upper bounds
 *             (K <= n, Es <= m).
 * Edges.      An int32 array of m (u, v) pairs, 8 bytes per edge, row-major.
 *             Undirected; each edge listed once; self-loops are allowed (they
 *             count twice toward their node's degree and never move labels or
 *             form superedges).  The pointer must be 16-byte aligned.
 * Determinism. Integer outputs are unique and bit-exact (independent of
 *             thread scheduling).  The ForceAtlas2 step is deterministic too:
 *             the tree's opening decisions use exact integer moments, and all
 *             sums run in a fixed order.
 */
#ifndef BGV_H
#define BGV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BGV_OK 0
#define BGV_EINVAL 1   /* bad size, null pointer, misaligned pointer or parameter */
#define BGV_ENOSPC 2   /* ws_bytes smaller than the *_ws_size query */
#define BGV_EDEVICE 3  /* the device reported an error (see the status word) */
#define BGV_ECUDA 4    /* a CUDA launch or copy failed */
#define BGV_ELIMIT 5   /* a size exceeds the fixed scratch of a no-allocation entry point */

/* Bits of the device status word. */
#define BGV_DEV_BADEDGE 1u     /* an edge endpoint outside [0, n) */
#define BGV_DEV_BADLABEL 2u    /* a label outside [0, n) */
/* bit 4u is unused: the Barnes-Hut traversal keeps no stack */
#define BGV_DEV_TIMEOUT 8u     /* a bounded device-side wait gave up */
#define BGV_DEV_BADHINT 16u    /* a sort hint entry outside [0, K) */

/* Library version, (major << 16) | minor. */
int bgv_version(void);

/* Human-readable name of a return code. */
const char *bgv_strerror(int code);

/* Zero the 256-byte header (status word and counters) of a new workspace.
 * Call once per workspace before its first use (or zero-fill it yourself). */
int bgv_ws_init(void *ws, void *stream);

/* Synchronise `stream` and return the device status word of workspace `ws`
 * in *out (0 = no device error).  `clear` != 0 resets it to 0 afterwards. */
int bgv_status(void *ws, void *stream, uint32_t *out, int clear);

/* ------------------------------------------------------------------------
 * 1. Degree count-min sketch (Algorithm 2; Section 3.3; Section 4.1).
 *
 * Hash family: h_i(x) = ((a_i x + b_i) mod (2^31 - 1)) mod width, where row i
 * draws a_i = 1 + z1 mod (2^31 - 2) and b_i = z2 mod (2^31 - 1) from two
 * SplitMix64 outputs of state seed + i.
 * Every endpoint of every edge adds 1 to sketch[i][h_i(endpoint)] for all
 * rows i; then deg_est[v] = min_i sketch[i][h_i(v)] (never below the true
 * degree).
 *   edges    [m][2] int32, 16-byte aligned      (in)
 *   sketch   [rows][width] uint32, row-major     (out)
 *   deg_est  [n] uint32                          (out)
 * Limits: 0 <= m < 2^31, 1 <= n < 2^31 - 1, 1 <= rows <= 16, 1 <= width.
 * ---------------------------------------------------------------------- */
size_t bgv_sketch_degrees_ws_size(int64_t m, int32_t n, int32_t rows, int32_t width);
int bgv_sketch_degrees(const int32_t *edges, int64_t m, int32_t n, int32_t rows, int32_t width,
                       uint64_t seed, uint32_t *sketch, uint32_t *deg_est,
                       void *ws, size_t ws_bytes, void *stream);

/* The same degree sketch for callers that cannot allocate device memory
 * (for example code running while a stream is captured, or a plugin whose
 * host application owns all device memory).  The paper has no counterpart:
 * this entry point only changes where the scratch lives.  The per-node
 * degree counters sit in a fixed array of device memory inside the library
 * (at most 4,194,304 nodes, 16 MiB, held by every GPU that loads the
 * library until exit) instead of a caller workspace; larger n returns
 * BGV_ELIMIT.  The first call on each device looks up the array's device
 * address (make it before any stream capture); every call clears the
 * counters, and all calls on a device share them, so calls whose work can
 * overlap on the GPU race and must be ordered on one stream.  Device-detected
 * bad edges are OR-ed into *status (device uint32).  status may be NULL:
 * the call then uses a status word of its own (cleared on every call),
 * synchronises `stream` at its end and returns BGV_EDEVICE if the device
 * found a bad edge.  Arguments otherwise as bgv_sketch_degrees. */
int bgv_sketch_degrees_noalloc(const int32_t *edges, int64_t m, int32_t n, int32_t rows, int32_t width,
                               uint64_t seed, uint32_t *sketch, uint32_t *deg_est, uint32_t *status,
                               void *stream);

/* ------------------------------------------------------------------------
 * 2. Community rounds (Algorithm 3; Section 3.2.1; Section 4.2.2).
 *
 * labels[v] = v and d[v] = deg_est[v] to start; D = threshold (0 means the
 * average degree floor(2m / n), Algorithm 3's first line).  Each of `passes`
 * rounds reads labels and degrees as they stood at the start of the round.
 * An edge (u, v), u != v, is skipped unless d[u] <= D and d[v] <= D and the
 * labels differ; the endpoint with the smaller degree is proposed to take
 * the other's label; on equal degrees nothing happens (tie_mode 0) or the
 * lower id takes the higher id's label (tie_mode 1).  At the end of the
 * round each node with proposals takes the one from the lowest edge index
 * and its degree grows by 1 (saturating).  Then D = min(D * growth, 2^32-1);
 * growth 0 multiplies by the first round's D instead, so round i uses D^i
 * (the delta^i schedule of Section 4.2.2).
 *   deg_est  [n] uint32 (in)     labels [n] int32 (out)
 *   deg_out  [n] uint32 (out, optional: final degrees, may be NULL)
 * Limits: passes >= 0, tie_mode in {0, 1}.
 * ---------------------------------------------------------------------- */
size_t bgv_communities_ws_size(int64_t m, int32_t n);
int bgv_communities(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est,
                    int32_t passes, uint32_t threshold, uint32_t growth, int32_t tie_mode,
                    int32_t *labels, uint32_t *deg_out, void *ws, size_t ws_bytes, void *stream);

/* Variants of the rounds.  threshold_mode 1 with threshold 0 starts from the
 * mode degree (Section 4.2.2 follows SCoDA in taking the most common degree):
 * the most frequent nonzero value of deg_est, ties to the smaller, computed
 * on the device and read back once (the call synchronises `stream` then).
 * (bgv_layout with threshold_mode 1 takes the mode of the exact degrees,
 * which it counts anyway for the sketch.)
 * jumps (0..64) synchronous pointer-jumping steps follow every round: each
 * label becomes its label's label, all read before the step.  The first
 * round's threshold is returned in *threshold_out (host, may be NULL).
 * Other arguments as bgv_communities. */
size_t bgv_communities_ex_ws_size(int64_t m, int32_t n);
int bgv_communities_ex(const int32_t *edges, int64_t m, int32_t n, const uint32_t *deg_est, int32_t passes,
                       uint32_t threshold, uint32_t growth, int32_t tie_mode, int32_t threshold_mode, int32_t jumps,
                       int32_t *labels, uint32_t *deg_out, uint32_t *threshold_out, void *ws, size_t ws_bytes,
                       void *stream);

/* Mode degree of deg [n] (device uint32): the most frequent value among the
 * nonzero ones, ties to the smaller, 0 if all are 0; returned in *mode_out
 * (host).  Synchronises `stream`. */
size_t bgv_mode_degree_ws_size(int32_t n);
int bgv_mode_degree(const uint32_t *deg, int32_t n, uint32_t *mode_out, void *ws, size_t ws_bytes, void *stream);

/* Modularity of a labelling (the quality the paper reports for its
 * communities, Table 1 column M): Q = sum over labels c of in_c / 2m -
 * (vol_c / 2m)^2, in_c twice the edges with both endpoints labelled c, vol_c
 * the number of endpoints labelled c.  Counted as exact integers and
 * combined in one FP64 division, so Q does not depend on thread order.
 * labels [n] int32 (device, values in [0, n)); *q_out host double.
 * Synchronises `stream`. */
size_t bgv_modularity_ws_size(int32_t n);
int bgv_modularity(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels, double *q_out, void *ws,
                   size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * 3. Supergraph (Section 4.1; Algorithm 3, "compute community sizes" and
 *    ForceAtlas2(Csrc, Cdst, Csize)).
 *
 * Supernodes are the distinct labels numbered in ascending label order:
 * node_map[v] = rank of labels[v]; *K_dev = number of distinct labels.
 * Superedges: the multiset {(min(map u, map v), max(...)) : labels[u] !=
 * labels[v]} sorted ascending and collapsed: ssrc[s] < sdst[s], sw[s] =
 * multiplicity; *Es_dev = count.  Community size: a count-min sketch (same
 * hash family, rows, width, seed) where every node v adds deg_est[v] at
 * h_i(labels[v]); mass[k] = 1 + min_i over the sketch at h_i(label of k),
 * saturated at 2^32 - 1.  Symmetric CSR: csr_off[K+1]; row k lists its
 * neighbours in ascending order in csr_adj with weights csr_w.
 *   node_map [n] int32;  ssrc, sdst [m] int32; sw [m] uint32;
 *   mass [n] uint32; csr_off [n+1] int32; csr_adj [2m] int32;
 *   csr_w [2m] uint32; K_dev, Es_dev: one int64 each.
 *   Optional (NULL allowed): vol [n] uint64 (exact sum of deg_est per
 *   supernode), count [n] uint32 (nodes per supernode), comm_label [n] int32
 *   (the label of each supernode).
 * Entries past K / Es / 2 Es / K+1 are left undefined.
 * ---------------------------------------------------------------------- */
size_t bgv_supergraph_ws_size(int64_t m, int32_t n, int32_t rows, int32_t width);
int bgv_supergraph(const int32_t *edges, int64_t m, int32_t n, const int32_t *labels,
                   const uint32_t *deg_est, int32_t rows, int32_t width, uint64_t seed,
                   int32_t *node_map, int64_t *K_dev, int32_t *ssrc, int32_t *sdst, uint32_t *sw,
                   int64_t *Es_dev, uint32_t *mass, int32_t *csr_off, int32_t *csr_adj,
                   uint32_t *csr_w, uint64_t *vol, uint32_t *count, int32_t *comm_label,
                   void *ws, size_t ws_bytes, void *stream);

/* Whole-graph CSR for ForceAtlas2 on the graph itself (Section 4.1: a layout
 * of the whole graph, coloured by the detected communities).  Row v lists
 * the distinct neighbours of v in ascending order; csr_w is the number of
 * edges joining the pair (1 for a simple graph); self-loops are ignored;
 * mass[v] = (number of distinct neighbours) + 1 (FA2's deg + 1).
 *   csr_off [n+1] int32, csr_adj [2m] int32, csr_w [2m] uint32, mass [n]
 *   uint32; *nnz_dev (device int64) receives csr_off[n]. */
size_t bgv_graph_csr_ws_size(int64_t m, int32_t n);
int bgv_graph_csr(const int32_t *edges, int64_t m, int32_t n, int32_t *csr_off, int32_t *csr_adj, uint32_t *csr_w,
                  uint32_t *mass, int64_t *nnz_dev, void *ws, size_t ws_bytes, void *stream);

/* Supernode colour groups (Section 4.3).  Communities are ordered by size
 * ascending (ties by index); group 0 (drawn brown) is the longest prefix of
 * that order whose sizes sum to at most half of the total; the remaining R
 * communities get group 1 + floor(10 * rank / R), small to big (the paper's
 * ten named colours).  sizes [K] uint32 (in, e.g. supernode masses),
 * group [K] uint8 (out).  Optionally (node_colour != NULL) every node v of a
 * whole-graph drawing takes its supernode's colour:
 * node_colour[v] = group[node_map[v]] for node_map [n] int32. */
size_t bgv_colour_groups_ws_size(int64_t K);
int bgv_colour_groups(int64_t K, const uint32_t *sizes, uint8_t *group, int32_t n, const int32_t *node_map,
                      uint8_t *node_colour, void *ws, size_t ws_bytes, void *stream);

/* Drawing: discs of radius[k] (sqrt of the size, Section 4.1) at xy[k] in
 * the colour of group[k] (Section 4.3: 0 brown, 1..10 light purple, purple,
 * light orange, orange, light red, red, light green, green, light blue,
 * blue), into rgba [H][W][4] uint8 (device, row-major, 4-byte aligned,
 * background white, alpha 255).  The discs' bounding box maps to the image
 * with one scale s = min(W, H) / largest extent from its low corner; pixel
 * (px, py) takes the disc whose scaled circle covers (px + 0.5, py + 0.5);
 * where discs overlap the smaller radius wins, then the smaller index.
 * Coverage is decided in FP32 with round-to-nearest steps.  W, H <= 32768. */
size_t bgv_render_ws_size(int32_t W, int32_t H);
int bgv_render(int64_t K, const float *xy, const float *radius, const uint8_t *group, int32_t W, int32_t H,
               uint8_t *rgba, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * 4. ForceAtlas2 (Section 3.1; Algorithm 1; the force model and adaptive
 *    speed of Jacomy et al. 2014 that the paper's implementation follows).
 *
 * Forces on supernode i with mass m_i (FP32):
 *   repulsion  kr m_i m_j (p_i - p_j) / |p_i - p_j|^2 summed over Barnes-Hut
 *              cells and leaf bodies (zero for coincident points);
 *   attraction -sum_j w_ij (p_i - p_j) over CSR neighbours;
 *   gravity    -kg m_i p_i / |p_i| (strong_gravity: -kg m_i p_i).
 * Step: swing_i = |F_i - Fprev_i|, traction_i = |F_i + Fprev_i| / 2;
 * S = sum m_i swing_i, T = sum m_i traction_i over the FP32 per-node
 * products, summed exactly (integer fixed-point accumulation) and rounded
 * once to FP64, so they are the correctly rounded sums whatever the thread
 * order (batched: per graph); if S > 0,
 * speed += min(tau T / S - speed, speed / 2); then
 * s_i = ks speed / (1 + speed sqrt(swing_i)), capped at ksmax / |F_i|;
 * p_i += s_i F_i; Fprev = F.
 * Quadtree: frame lo = min p, side = max extent * (1 + 2^-20); body fixed
 * point U = trunc((p - lo) / side * 2^32); Morton key over the top
 * max_depth bits of U; a cell splits while it holds more than leaf_cap
 * bodies and is above max_depth.  A cell containing the body is opened; a
 * leaf is summed body by body; otherwise the cell is accepted iff
 * (side 2^-level)^2 < theta^2 |p_i - c|^2, all in FP32, where c is the
 * cell's centre of mass from exact integer moments of U.
 * Layout: pos, F, Fprev are [K][2] float (x, y interleaved), 8-byte aligned.
 * ---------------------------------------------------------------------- */
typedef struct bgv_fa2_params {
    float theta;            /* Barnes-Hut opening parameter (1.2) */
    float kr;               /* repulsion scaling (2.0; the paper's runs used 80) */
    float kg;               /* gravity (1.0) */
    float tau;              /* jitter tolerance (1.0) */
    float ks;               /* local speed constant (0.1) */
    float ksmax;            /* local speed cap constant (10.0) */
    int32_t strong_gravity; /* 0 or 1 (0) */
    int32_t leaf_cap;       /* bodies per leaf, >= 1 (1) */
    int32_t max_depth;      /* quadtree levels, 1..24 (24) */
    int32_t reserved;       /* must be 0 */
    uint64_t seed;          /* initial positions (1) */
} bgv_fa2_params;

/* Per-step statistics kept in the FA2 workspace. */
typedef struct bgv_fa2_stats {
    double S;                   /* sum of m_i swing_i, last step */
    double T;                   /* sum of m_i traction_i, last step */
    uint64_t interactions;      /* body-cell plus body-body terms, last step */
    uint64_t tree_nodes;        /* quadtree internal nodes, last step */
    uint64_t interactions_total;/* terms summed over all steps since bgv_ws_init */
    uint64_t steps_total;       /* steps completed since bgv_ws_init */
    uint32_t status;            /* device status word */
    uint32_t reserved;
} bgv_fa2_stats;

void bgv_fa2_default_params(bgv_fa2_params *p);

/* Initial state: pos[i] per axis = U * 2 R - R with R = sqrt(K) and U the top
 * 24 bits of SplitMix64 at state seed + 2 i + axis (FP32); Fprev = 0;
 * *speed = 1 (device double). */
int bgv_fa2_init(int64_t K, const bgv_fa2_params *p, float *pos, float *Fprev, double *speed, void *stream);

/* Workspace for bodies K and CSR entries nnz.  Every FA2 call below takes
 * the same nnz, which must equal csr_off[K] (2 Es for a supergraph). */
size_t bgv_fa2_ws_size(int64_t K, int64_t nnz);

/* Forces only, at positions pos, without changing any state:
 * Fr, Fa, Fg [K][2] float (repulsion, attraction, gravity); any may be NULL. */
int bgv_fa2_forces(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                   const uint32_t *mass, const bgv_fa2_params *p, const float *pos,
                   float *Fr, float *Fa, float *Fg, void *ws, size_t ws_bytes, void *stream);

/* One iteration in place: F receives the total force, pos/Fprev/speed are
 * advanced.  Statistics of the step stay in `ws` (bgv_fa2_read_stats). */
int bgv_fa2_step(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                 const uint32_t *mass, const bgv_fa2_params *p, float *pos, float *F, float *Fprev,
                 double *speed, void *ws, size_t ws_bytes, void *stream);

/* `iterations` steps; with use_graph != 0 one step is captured into a CUDA
 * graph on `stream` and replayed (the stream must not be capturing). */
int bgv_fa2_run(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                const uint32_t *mass, const bgv_fa2_params *p, int32_t iterations, int32_t use_graph,
                float *pos, float *F, float *Fprev, double *speed, void *ws, size_t ws_bytes, void *stream);

/* Profiling form of bgv_fa2_run: `iterations` steps launched one by one
 * (no graph) with CUDA events recorded at the boundaries of the
 * BGV_FA2_STAGES stages of each step (on the library stream that runs the
 * main chain); synchronises `stream` and returns in stage_ms[BGV_FA2_STAGES]
 * the summed milliseconds per stage:
 *   0 frame + Morton keys (from the second step on: frame + the hinted
 *   sort's samples), 1 sort (the radix sort in the first step, the rest of
 *   the hinted sort in the others), 2 gather into Morton order and moment
 *   prefix sums, 3 radix tree and quadtree cells, 4 pre-order layout,
 *   5 Barnes-Hut repulsion, 6 the wait for the attraction (which runs beside
 *   stages 0-5), 7 total force, swing/traction, speed and displacement (one
 *   persistent kernel).
 * Creates and destroys (BGV_FA2_STAGES + 1) * iterations CUDA events. */
#define BGV_FA2_STAGES 8
int bgv_fa2_run_timed(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                      const uint32_t *mass, const bgv_fa2_params *p, int32_t iterations, float *pos, float *F,
                      float *Fprev, double *speed, void *ws, size_t ws_bytes, void *stream, float *stage_ms);

/* Number of kernel launches this library has issued in the process so far
 * (a kernel replayed from a CUDA graph counts once per replay). */
uint64_t bgv_launch_count(void);

/* Synchronise `stream` and copy the statistics of the last step. */
int bgv_fa2_read_stats(void *ws, void *stream, bgv_fa2_stats *out);

/* ------------------------------------------------------------------------
 * 5. The whole pipeline (Algorithm 3 end to end): sketch, rounds,
 *    supergraph, initial positions and `iterations` ForceAtlas2 steps.
 * ---------------------------------------------------------------------- */
typedef struct bgv_layout_params {
    int32_t rows;        /* sketch rows (4) */
    int32_t width;       /* sketch columns (4096) */
    uint64_t seed;       /* hash seed (1) */
    int32_t passes;      /* community rounds (3) */
    uint32_t threshold;  /* degree threshold; 0 = floor(2m / n) (0) */
    uint32_t growth;     /* threshold factor per round; 0 = the first threshold (delta^i) (2) */
    int32_t tie_mode;    /* 0 or 1 (0) */
    int32_t threshold_mode; /* with threshold 0: 0 = floor(2m / n), 1 = the graph's most common degree (0) */
    int32_t jumps;       /* pointer-jumping steps after every round, 0..64 (0) */
    int32_t iterations;  /* ForceAtlas2 steps (200) */
    int32_t use_graph;   /* replay the FA2 step as a CUDA graph (1) */
    bgv_fa2_params fa2;
} bgv_layout_params;

void bgv_layout_default_params(bgv_layout_params *p);

/* Workspace for the device pipeline; it holds every intermediate
 * (sketch, degrees, labels, supergraph, CSR, FA2 state and scratch). */
size_t bgv_layout_ws_size(int64_t m, int32_t n, const bgv_layout_params *p);

/* Device pipeline.  Synchronises `stream` once, after the supergraph, to
 * learn K and Es (returned in *K_out, *Es_out, host int64), and once at the
 * end.  Outputs: node_map [n] int32 (supernode of every node), xy [n][2]
 * float (first K rows valid), radius [n] float (sqrt of mass, first K
 * valid).  Returns BGV_EDEVICE if the device reported a bad edge. */
int bgv_layout(const int32_t *edges, int64_t m, int32_t n, const bgv_layout_params *p,
               int32_t *node_map, float *xy, float *radius, int64_t *K_out, int64_t *Es_out,
               void *ws, size_t ws_bytes, void *stream);

/* The same pipeline from HOST memory: copies h_edges (pinned memory
 * recommended) into the workspace, runs bgv_layout, copies node_map, xy and
 * radius back to the host arrays, and synchronises `stream`. */
int bgv_layout_host(const int32_t *h_edges, int64_t m, int32_t n, const bgv_layout_params *p,
                    int32_t *h_node_map, float *h_xy, float *h_radius, int64_t *K_out, int64_t *Es_out,
                    void *ws, size_t ws_bytes, void *stream);

/* Workspace for bgv_layout_host: bgv_layout_ws_size plus room for the edges
 * and the outputs. */
size_t bgv_layout_host_ws_size(int64_t m, int32_t n, const bgv_layout_params *p);

/* ------------------------------------------------------------------------
 * 6. Batched form: G independent graphs laid out in one pass of every
 *    stage (Algorithm 3 applied to each graph; the paper runs its tables
 *    graph by graph, so this entry point has no counterpart there).  The
 *    result for every graph is the one bgv_layout gives for it alone: the
 *    integer stages (node_map, supernode and superedge counts) exactly, the
 *    positions up to FP32 summation order, because graph g keeps its own
 *    sketch matrices (rows x width each, local node ids hashed), its own
 *    degree threshold (floor(2 m_g / n_g) when p->threshold is 0), its own
 *    community-size sketch, quadtree frame, initial square, and speed.
 *
 * Host arrays: edge_off [G+1] int64 and node_off [G+1] int32, both
 * starting at 0; graph g has node_off[g+1] - node_off[g] >= 1 nodes and
 * the edges edges[edge_off[g] .. edge_off[g+1]) as (u, v) int32 pairs of
 * LOCAL ids 0 .. n_g - 1.  An endpoint outside its graph sets
 * BGV_DEV_BADEDGE and the call returns BGV_EDEVICE.  Totals must fit the
 * single-graph limits (N < 2^31 - 1 nodes, m < 2^31 edges).
 * Outputs (device): node_map [N] int32 -- the LOCAL supernode id of every
 * node; xy [N][2] float and radius [N] float, graph g's supernodes in rows
 * K_off[g] .. K_off[g+1] (first K_off[G] rows valid).  Host outputs:
 * K_off [G+1], Es_off [G+1] int64, the supernode and superedge offsets.
 * Synchronises `stream` after the supergraph and at the end.
 * ---------------------------------------------------------------------- */
size_t bgv_layout_batched_ws_size(int32_t G, const int64_t *edge_off, const int32_t *node_off,
                                  const bgv_layout_params *p);
int bgv_layout_batched(const int32_t *edges, int32_t G, const int64_t *edge_off, const int32_t *node_off,
                       const bgv_layout_params *p, int32_t *node_map, float *xy, float *radius,
                       int64_t *K_off, int64_t *Es_off, void *ws, size_t ws_bytes, void *stream);

/* Batched ForceAtlas2 on caller supergraphs: bodies of graph g are rows
 * koff[g] .. koff[g+1] (host int64 [G+1], strictly increasing, koff[0] = 0,
 * K = koff[G]) and the CSR (K rows, nnz entries, global row ids) must not
 * link two graphs.  Each graph gets its own frame, initial square (R =
 * sqrt(K_g), local index in the SplitMix64 state), and speed: speed is
 * [G] device double.  The offsets are copied into `ws` on every call. */
size_t bgv_fa2_ws_size_batched(int32_t G, int64_t K, int64_t nnz);
int bgv_fa2_init_batched(int32_t G, const int64_t *koff, const bgv_fa2_params *p, float *pos, float *Fprev,
                         double *speed, void *ws, size_t ws_bytes, void *stream);
int bgv_fa2_forces_batched(int32_t G, const int64_t *koff, int64_t nnz, const int32_t *csr_off,
                           const int32_t *csr_adj, const uint32_t *csr_w, const uint32_t *mass,
                           const bgv_fa2_params *p, const float *pos, float *Fr, float *Fa, float *Fg,
                           void *ws, size_t ws_bytes, void *stream);
int bgv_fa2_run_batched(int32_t G, const int64_t *koff, int64_t nnz, const int32_t *csr_off,
                        const int32_t *csr_adj, const uint32_t *csr_w, const uint32_t *mass,
                        const bgv_fa2_params *p, int32_t iterations, int32_t use_graph, float *pos, float *F,
                        float *Fprev, double *speed, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * 7. Autotuners.  The radix sort of the supergraph and ForceAtlas2 stages
 *    runs either as one onesweep kernel per pass with decoupled look-back
 *    (method 0), 8 keys per thread up to a size cutoff and 16 above it, or
 *    as one cooperative kernel for all its passes (method 1: per pass, digit
 *    counts per block chunk, a scan over the chunks, a stable scatter; no
 *    look-back), or by size (method 2, the default): cooperative for keys
 *    with values in a range of counts and for keys alone from its lower
 *    end up, onesweep otherwise.  bgv_autotune_sort times all
 *    three forms on this GPU for 2^14, 2^16, ... <= max_keys keys (48-bit
 *    keys with 32-bit values, SplitMix64 of the index), sets the cutoff to
 *    the largest size at which 8 was not slower, and the cooperative range
 *    to the span of sizes where it was faster (method 0 if none).  All are
 *    process wide; they start at a cutoff of 2^40 (8 keys per thread at every
 *    size) and a cooperative range of [2^21, 2^23] (keys alone: from 2^21
 *    up), as measured on GB300;
 *    workspaces stay valid whatever they are.  bgv_set_sort_cutoff and
 *    bgv_set_sort_method (0, 1, 2) set them directly and return the previous
 *    value.
 *    Synchronises `stream` once per timed sort.  The paper has no
 *    counterpart.
 * ---------------------------------------------------------------------- */
typedef struct bgv_tune_report {
    int32_t count;          /* sizes timed */
    int32_t sizes_log2[9];  /* log2 of each size */
    float ms8[9];           /* median milliseconds, onesweep, 8 keys per thread */
    float ms16[9];          /* median milliseconds, onesweep, 16 keys per thread */
    float ms_coop[9];       /* median milliseconds, cooperative sort */
    int32_t method;         /* the method now in force: 0, 1 or 2 (by size) */
    int64_t cutoff;         /* the cutoff now in force */
    int64_t coop_lo, coop_hi; /* key counts sorted cooperatively under method 2 */
} bgv_tune_report;

/* bgv_autotune_fa2 picks the launch shapes of the ForceAtlas2 step on the
 * caller's supergraph: the longest CSR rows the attraction sums one lane
 * each (8, 16, 32; longer rows take a warp each, or a block above 4,096
 * entries), the threads per block of the Barnes-Hut traversal (128, 256) and
 * the blocks per SM of the persistent tail kernel (2, 4, 8; capped at what
 * stays resident).  One shape at a time, it times whole steps (the median of
 * three after a warm-up step) from positions `pos` (device, not changed:
 * steps run on a copy in `ws`, with Fprev = 0 and speed 1), keeps the
 * fastest, and leaves the choice in force for the process.  The traversal
 * and tail shapes do not change any result; the row split of the attraction
 * changes the grouping of some FP32 row sums (within rounding).
 * Synchronises `stream`.  bgv_set_fa2_tune sets the shapes directly
 * (BGV_EINVAL for other values). */
typedef struct bgv_fa2_tune_report {
    int32_t att_short;          /* chosen: longest rows summed one lane each */
    int32_t repulse_threads;    /* chosen threads per block of the traversal */
    int32_t tail_blocks_per_sm; /* chosen blocks per SM of the step's tail */
    int32_t reserved;
    float ms_att_short[3];      /* median step ms at 8, 16, 32 */
    float ms_repulse_threads[2];/* at 128, 256 threads */
    float ms_tail_blocks[3];    /* at 2, 4, 8 blocks per SM */
} bgv_fa2_tune_report;

size_t bgv_autotune_fa2_ws_size(int64_t K, int64_t nnz);
int bgv_autotune_fa2(int64_t K, int64_t nnz, const int32_t *csr_off, const int32_t *csr_adj, const uint32_t *csr_w,
                     const uint32_t *mass, const bgv_fa2_params *p, const float *pos, bgv_fa2_tune_report *out,
                     void *ws, size_t ws_bytes, void *stream);
int bgv_set_fa2_tune(int32_t att_short, int32_t repulse_threads, int32_t tail_blocks_per_sm);

size_t bgv_autotune_sort_ws_size(int64_t max_keys);
int bgv_autotune_sort(int64_t max_keys, bgv_tune_report *out, void *ws, size_t ws_bytes, void *stream);
int64_t bgv_sort_cutoff(void);
int64_t bgv_set_sort_cutoff(int64_t cutoff);
int32_t bgv_set_sort_method(int32_t method);

/* ------------------------------------------------------------------------
 * Hinted sort.  The radix tree of the Barnes-Hut repulsion (§3.1, the
 * quadtree of ForceAtlas2's repulsion) is built over the bodies in Morton
 * order.  A body moves little between two steps, so from the second step of
 * a run on (bgv_fa2_run, bgv_layout*) the library finds that order with a
 * sample sort whose buckets follow the previous step's order, instead of a
 * full radix sort; both give the same order, (key, id).  The paper has no
 * counterpart.
 *
 * bgv_sort_hinted sorts the pairs (keys[id], id), id in [0, K), into (key, id)
 * order and writes them to out_keys and out_ids.  `hint` is an order of the
 * ids (a permutation of [0, K)) that only guides the work: the closer it is
 * to the sorted order, the more even the buckets.  keys: device, K uint64;
 * hint: device, K uint32; out_keys/out_ids: device, K entries each, aliasing
 * neither input nor each other; keys and out_keys 8-byte aligned, hint and
 * out_ids 4-byte aligned, ws 256-byte aligned (BGV_EINVAL otherwise).  0 <= K <=
 * bgv_sort_hinted_max_keys() (4,194,304; BGV_EINVAL above).  A hint entry
 * >= K raises BGV_DEV_BADHINT in the workspace's status word and is read as
 * 0, and the call returns BGV_EDEVICE; a hint with a repeated id gives an
 * unspecified order but no access outside the arrays.  Synchronises
 * `stream`.  ws: bgv_sort_hinted_ws_size(K) bytes (0 for a K out of range),
 * header zeroed by bgv_ws_init.
 *
 * bgv_set_fa2_order(1) (the default) makes ForceAtlas2 runs use the hinted
 * sort from their second step on (for K up to the same limit); 0 makes every
 * step use the full radix sort.  Process wide; returns the previous value
 * (-1 and no change for other values).  A CUDA graph captured earlier keeps
 * the method it was captured with.
 * ---------------------------------------------------------------------- */
int64_t bgv_sort_hinted_max_keys(void);
size_t bgv_sort_hinted_ws_size(int64_t K);
int bgv_sort_hinted(const uint64_t *keys, const uint32_t *hint, int64_t K, uint64_t *out_keys, uint32_t *out_ids,
                    void *ws, size_t ws_bytes, void *stream);
int32_t bgv_set_fa2_order(int32_t method);

/* ------------------------------------------------------------------------
 * 8. Bounded waits.  Every decoupled look-back wait in the library (radix
 *    sort passes, the ForceAtlas2 moment pass, the CSR pass of the
 *    supergraph) polls at most `limit` rounds for a predecessor tile, then
 *    sets BGV_DEV_TIMEOUT in the status word and lets its block finish, so a
 *    wait that cannot end is reported instead of hanging the GPU.  The paper
 *    has no counterpart: this is the library's own failure detection.
 *
 * bgv_set_spin_limit sets the bound for the process (limit >= 0; default
 * 2^22 rounds, a few seconds) and returns the previous one (-1 and no
 * change for a negative limit).  A CUDA graph captured earlier keeps the
 * bound it was captured with.
 *
 * bgv_check_wait_timeout runs one block of look-back kernel `which` (0 a
 * radix-sort pass, 1 the moment pass, 2 the CSR pass) as the second tile of
 * a two-tile input whose first tile never runs, so its wait cannot end and
 * must give up at the bound: afterwards the status word of `ws` holds
 * BGV_DEV_TIMEOUT.  Synchronises `stream`.  ws: a workspace of
 * bgv_check_wait_timeout_ws_size() bytes (header zeroed, see bgv_ws_init).
 * ---------------------------------------------------------------------- */
int32_t bgv_set_spin_limit(int32_t limit);
size_t bgv_check_wait_timeout_ws_size(void);
int bgv_check_wait_timeout(int32_t which, void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BGV_H */
