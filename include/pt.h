/*
 * pt.h -- C ABI of the GB300 P3T long-range force library (libpt.so).
 *
 * The library computes the long-range half of the P3T Hamiltonian split used
 * by PeTar (Wang, Iwasawa, Nitadori & Makino 2020):
 *
 *   Sec. 5.1, Eq. 11:  H_L = -sum_{i<j} G m_i m_j (1 - W(r_ij)) / r_ij
 *   Sec. 6.1, Eqs. 15-17: W(x), K(x) with x = (r - r_in)/(r_out - r_in)
 *
 * so that for every particle i
 *
 *   a_i   = G sum_j m_j (x_j - x_i) (1 - K(x_ij)) / r_ij^3
 *   phi_i = -G sum_j m_j (1 - W(x_ij)) / r_ij       (j != i)
 *
 * with distant particles grouped into Barnes-Hut cells "inside theta"
 * (Sec. 4; Sec. 5.1, Fig. 2) that act through their monopole and quadrupole
 * (Sec. 6.4.2, Eqs. 30-31), and it returns the r_out neighbour lists that the
 * short-range integrator consumes (Sec. 6, Fig. 3 step 2).
 *
 * Pipeline on one GPU (every step is a CUDA kernel of this library):
 *   root box and 63-bit Morton keys -> LSD radix sort -> octree topology ->
 *   bottom-up multipoles -> groups -> group-wise walk (cell and particle
 *   lists) -> force kernel (FP64 or FP32-mixed) with fused neighbour
 *   extraction -> neighbour CSR -> energy and momentum sums.
 *
 * The tree, group and walk definitions are fixed exactly (the paper does not
 * define them); they are identical to the project's CPU oracle:
 *   grid     q_d = clamp(floor((x_d - o_d) * 2^21 / S), 0, 2^21-1), o = box
 *            minimum, S = largest box extent (1 if all points coincide);
 *   keys     bit 3b+2 / 3b+1 / 3b of the key = bit b of q_x / q_y / q_z;
 *   order    ascending key, ties by ascending original index;
 *   nodes    level-l node = maximal run of sorted keys sharing the top 3l
 *            bits; it is a leaf if it holds <= n_leaf particles or l = 21;
 *   groups   a node with <= n_group particles, or a leaf, is a group; larger
 *            nodes pack consecutive small children greedily (<= n_group);
 *   walk     cell C is accepted for group G iff s^2 < theta^2 d^2 (s = side
 *            of C's cube, d = distance from G's grid box to the cube centre,
 *            both in half grid cells, product in float64) and the squared
 *            gap between the grid boxes, in whole cells, is at least
 *            floor((r_out * 2^21 / S)^2) + 2 (so no pair closer than r_out
 *            is ever inside an accepted cell); otherwise leaves go to the
 *            particle-particle (PP) list and internal cells are opened (a
 *            leaf that passes the gap test is kept in the group's far PP
 *            segment, evaluated as plain Newtonian pairs);
 *   neighbours  j != i with dx*dx + dy*dy + dz*dz < r_out*r_out evaluated in
 *            float64 left to right without fused multiply-add.
 *
 * Conventions for every entry point:
 *   - Return value: PT_OK (0) or one of the PT_ERR_* codes below; no
 *     exception crosses the ABI.  pt_last_error() gives a message.
 *   - Pointers may be device memory (cudaMalloc / torch tensors) or host
 *     memory; the library detects which.  Host buffers are staged through
 *     device memory inside the call.  The caller owns every buffer it passes.
 *   - All work is ordered on the context's stream.  Calls that return counts
 *     (pt_tree_build, pt_longrange_force, pt_batch_longrange_force)
 *     synchronise that stream before returning.  pt_longrange_force copies
 *     host outputs (acc, pot) on a private stream of the context that waits
 *     for the force kernel; it is synchronised before the call returns.
 *   - Layouts: positions are n x 3 float64, row-major (x, y, z per particle);
 *     masses n float64 (>= 0); accelerations n x 3 float64; potentials n
 *     float64; every output is in the caller's original particle order.
 *   - The library owns its workspace (tree arrays, lists); it is sized on
 *     first use and reused by later calls with the same or smaller sizes.
 *   - There is no CPU fallback: without a usable GPU every call fails with
 *     PT_ERR_CUDA.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define PT_OK            0
#define PT_ERR_ARG       1   /* bad argument: n < 1, theta < 0, r_in >= r_out,
                                r_in < 0, n_leaf < 1, n_group < 1, order not
                                0/2, non-finite position or negative mass   */
#define PT_ERR_OOM       2   /* device allocation failed                     */
#define PT_ERR_CAPACITY  3   /* nb_capacity too small; *nb_total holds the
                                number needed; acc and pot are valid         */
#define PT_ERR_TIMEOUT   4   /* a bounded device wait ran out                */
#define PT_ERR_CUDA      5   /* CUDA runtime error                           */
#define PT_ERR_INTERNAL  6   /* internal limit exceeded (message says which) */

/* ---- precision of the pair arithmetic ---- */
#define PT_FP64   0          /* everything in float64                        */
#define PT_MIXED  1          /* float64 storage, group-relative float32 pair
                                arithmetic with float-float accumulation     */

typedef struct pt_ctx pt_ctx;
typedef struct pt_tree pt_tree;

/* Force parameters (Sec. 6.1 and Sec. 7.1.1, Table 2 use theta 0.3/0.5,
 * quadrupole moments and r_out/r_in = 10).  r_in, r_out are the scalar
 * changeover radii (the mass-dependent radii of Eq. 12 set mass_dependent). */
typedef struct {
    double theta;        /* opening angle, >= 0 (0 = direct sum via PP)      */
    double r_in, r_out;  /* changeover radii, 0 <= r_in < r_out              */
    double G;            /* gravitational constant (1 in Henon units)        */
    int n_leaf;          /* max particles in a leaf (depth cap 21 aside)     */
    int n_group;         /* max particles in a walk group                    */
    int order;           /* 0 = monopole, 2 = monopole + quadrupole          */
    int precision;       /* PT_FP64 or PT_MIXED                              */
    int mass_dependent;  /* 1: per-particle radii s_i (r_in, r_out), a pair
                            using the larger (Sec. 6.1, Eqs. 12 and 16)      */
} pt_params;

/* Counters and sums of one force evaluation. */
typedef struct {
    int64_t n;                  /* particles                                 */
    int64_t nodes;              /* tree nodes                                */
    int64_t groups;             /* walk groups                               */
    int64_t max_level;          /* deepest tree level                        */
    int64_t cell_list_total;    /* sum over groups of cell-list lengths      */
    int64_t pp_list_total;      /* sum over groups of PP-list lengths        */
    int64_t cell_interactions;  /* sum over groups of n_G * cell-list length */
    int64_t pp_interactions;    /* sum over groups of n_G * PP-list length   */
    int64_t neighbours;         /* total neighbour-list entries              */
    double energy;              /* sum_i (1/2) m_i phi_i, float64            */
    double momentum[3];         /* sum_i m_i a_i, float64                    */
    double ms_build;            /* GPU time of the last tree build           */
    double ms_walk;             /* GPU time of the walk                      */
    double ms_force;            /* GPU time of the force kernel              */
    double ms_total;            /* GPU time of the force call (walk..sums)   */
    int64_t pp_changeover_interactions; /* mixed path: PP interactions evaluated
                                   with the changeover (a warp takes that path
                                   when any of its pairs is within r_out); the
                                   others used the plain Newtonian pair, which
                                   is exact beyond r_out (K = W = 0)         */
    int64_t max_walk_stack;     /* deepest walk stack (pending nodes per warp) */
    int64_t launches_build;     /* kernels launched by the last tree build   */
    int64_t launches_force;     /* kernels launched by the force call        */
} pt_stats;

/* Creates a context on CUDA device `device`, ordering all work on `stream`
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).
 * *ctx receives the handle; destroy it with pt_ctx_destroy. */
int pt_ctx_create(pt_ctx **ctx, int device, void *stream);

/* Frees the context's workspace (waits for its stream first).  Trees built
 * in this context that are still alive lose their device memory and become
 * empty handles: pass them to pt_tree_free (which then only releases the
 * handle) or rebuild them with pt_tree_build in another context. */
int pt_ctx_destroy(pt_ctx *ctx);

/* Message of the last failing call on ctx (static storage in ctx). */
const char *pt_last_error(const pt_ctx *ctx);

/* Builds keys, sort order, octree, multipoles and groups for n particles
 * (pos n x 3, mass n; host or device).  The tree keeps its own copies and
 * the parameters; *tree receives it (reuse: pass the same *tree again to
 * rebuild in place when its previous size suffices, else a new one is
 * made).  Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA, PT_ERR_INTERNAL. */
int pt_tree_build(pt_ctx *ctx, int64_t n, const double *pos, const double *mass,
                  const pt_params *params, pt_tree **tree);

/* As pt_tree_build, with mass-dependent changeover radii (Sec. 6.1, Eq. 12):
 * particle i has radii s_i (r_in, r_out) and a pair uses the larger pair
 * (Eq. 16), so the changeover, the walk's r_out gap and the neighbour lists all
 * use s_ij = max(s_i, s_j).  params->mass_dependent must be 1.  radius_scale
 * (n doubles, host or device, each >= 1 in the paper's use; a factor that is
 * not finite and positive returns PT_ERR_ARG) gives s_i; if it
 * is NULL the library computes Eq. 12, s_i = max(1, m_i / <m>)^(1/3) with <m>
 * the mean mass, on the device (CUDA cbrt: within 1 ulp of a host cbrt, so
 * pass the factors explicitly when neighbour lists must match a host
 * computation bit for bit). */
int pt_tree_build_scaled(pt_ctx *ctx, int64_t n, const double *pos, const double *mass,
                         const double *radius_scale, const pt_params *params, pt_tree **tree);

/* Walks the tree, evaluates acc (n x 3) and pot (n), both in the caller's
 * particle order, and, if nb_offsets is not NULL, the r_out neighbour lists
 * as CSR: nb_offsets (n+1 int64) and nb_idx (nb_capacity int32 original
 * indices, ascending within each row).  *nb_total (if not NULL) receives
 * the number of entries.  If nb_capacity is too small the call returns
 * PT_ERR_CAPACITY with acc, pot and *nb_total valid and the CSR untouched.
 * stats may be NULL. */
int pt_longrange_force(pt_ctx *ctx, pt_tree *tree, double *acc, double *pot,
                       int64_t *nb_offsets, int32_t *nb_idx, int64_t nb_capacity,
                       int64_t *nb_total, pt_stats *stats);

/* Releases a tree (waits for its context's stream first, if the context
 * still exists). */
int pt_tree_free(pt_tree *tree);

/* One independent particle set in a batch. */
typedef struct {
    int64_t n;               /* particles (>= 1)                              */
    const double *pos;       /* n x 3                                         */
    const double *mass;      /* n                                             */
    double r_in, r_out;      /* this set's changeover radii                   */
    double *acc;             /* out: n x 3                                    */
    double *pot;             /* out: n                                        */
    int64_t *nb_offsets;     /* out: n+1, or NULL for no neighbour lists      */
    int32_t *nb_idx;         /* out: nb_capacity entries (cluster-local ids)  */
    int64_t nb_capacity;
    int64_t nb_total;        /* out: entries needed                           */
    const double *radius_scale;  /* n radius factors (mass_dependent) or NULL;
                                    each finite and > 0, else PT_ERR_ARG     */
} pt_cluster_desc;

/* Evaluates n_clusters independent sets in one pass of the pipeline: every
 * stage runs once over all sets (one forest with one root per set), so one
 * launch sequence serves the whole batch.  params->r_in/r_out are ignored in
 * favour of each descriptor's radii.  All descriptor pointers must be of the
 * same kind (all device or all host).  flags: PT_BATCH_GRAPH replays a CUDA
 * graph of the launch sequence when the batch shape repeats.  stats, if not
 * NULL, receives the totals over the batch. */
#define PT_BATCH_GRAPH 1
int pt_batch_longrange_force(pt_ctx *ctx, int n_clusters, pt_cluster_desc *desc,
                             const pt_params *params, int flags, pt_stats *stats);

/* Autotuner: evaluates the batch `desc` (one set is a batch of one) with every
 * (n_leaf, n_group) pair from the candidate lists, timing the device work of
 * the tree build and the force call (best of `reps` runs after one sizing
 * run), and writes the fastest parameters to *best (the other fields are
 * copied from *base) and its time in ms to *best_ms (may be NULL).  NULL or
 * empty lists select n_leaf in {4, 8, 16, 32} and n_group in
 * {32, 48, 64, 96, 128}.  Results are cached in the context per (number of
 * sets, power-of-two buckets of the total and mean set size, theta, order,
 * precision); a cached entry is returned without timing.  The descriptors'
 * outputs hold the last candidate's results.  The force kernel's lane layout
 * (targets per lane and sub-streams per warp) is chosen per group at run
 * time and needs no tuning. */
int pt_autotune(pt_ctx *ctx, int n_clusters, pt_cluster_desc *desc, const pt_params *base,
                const int *leaf_candidates, int n_leaf_candidates, const int *group_candidates,
                int n_group_candidates, int reps, pt_params *best, double *best_ms);

/* ---- serving: long-range kick requests from many resident simulations ---- */

/* A server keeps the particle state of many simulations resident on the
 * device and serves "drift, long-range force, kick" requests for them with
 * continuous batching: `workers` worker threads, each with its own context and
 * stream, take the queued requests in arrival order (at most one per
 * simulation, none for a simulation another worker has on the GPU, up to
 * max_batch_particles particles) and evaluate them in one pass of the
 * pipeline (pt_batch_longrange_force).  Requests that arrive while batches run
 * are taken by the next free worker, and the workers' batches overlap on the
 * device: with two or more workers, half of them serve the large simulations
 * on low-priority streams and the others the small ones on high-priority
 * streams, so small requests do not wait for a large simulation's batch.  A
 * simulation's requests run one after the other, in submission order.
 * Admission is checked against hbm_budget_bytes: the resident state of every
 * simulation (about 100 bytes plus neighbour capacity per particle) plus a
 * workspace reserve of 1,536 bytes per batch particle and worker must fit.
 * A request on simulation s does x += v dt_drift (a free drift standing in for
 * the short-range integrator, out of scope here), computes the long-range
 * acceleration and potential (and neighbour lists if requested) of s, and
 * then kicks v += a dt_kick (Sec. 6, Fig. 3, the P3T kick).  Its result is the
 * same alone and batched with others. */
typedef struct pt_server pt_server;

typedef struct {
    size_t hbm_budget_bytes;      /* device memory the server may use          */
    int64_t max_batch_particles;  /* particles per batch; 0 = from the budget  */
    int max_sims;                 /* simulations that may be resident          */
    int neighbours;               /* 1: keep r_out neighbour lists per sim     */
    pt_params params;             /* theta, G, n_leaf, n_group, order,
                                     precision (r_in / r_out come per sim)     */
    int workers;                  /* concurrent batch pipelines, 0 = 4, <= 16  */
    int64_t large_sim_particles;  /* with 2+ workers: simulations of at least
                                     this size go to the first half of the
                                     workers (low stream priority), the rest
                                     to the other half; 0 = 2^20             */
} pt_server_config;

typedef struct {
    int64_t ticket;
    int sim;
    int status;                   /* PT_OK or the batch's error code            */
    double t_submit, t_start, t_done;   /* seconds on the server's clock        */
    int batch_size;               /* requests served by the same batch          */
    int64_t batch_particles;
} pt_request_info;

typedef struct {
    int64_t batches, requests, particles, interactions;
    double busy_s, uptime_s;      /* time with a batch on the device, lifetime */
    int64_t resident_bytes, max_batch_particles, queued;
} pt_server_stats_t;

/* Starts a server (and its worker threads) on the calling thread's current
 * device, each worker with its own stream and context; max_batch_particles
 * 0 means min(2^22, the budget's share).  `ctx` must be a valid context (its
 * device is used for checks only).  Errors: PT_ERR_ARG, PT_ERR_OOM, PT_ERR_CUDA. */
int pt_server_create(pt_ctx *ctx, const pt_server_config *cfg, pt_server **srv);
/* Finishes the queued requests, stops the worker and frees all state. */
int pt_server_destroy(pt_server *srv);
/* Copies a simulation's n particles (pos, vel n x 3; mass n; host or device)
 * into resident device memory; *sim_id receives its id.  PT_ERR_CAPACITY if
 * the HBM budget, max_sims or max_batch_particles would be exceeded. */
int pt_server_add_sim(pt_server *srv, int64_t n, const double *pos, const double *vel,
                      const double *mass, double r_in, double r_out, int *sim_id);
/* Waits for the simulation's requests, then frees its state. */
int pt_server_remove_sim(pt_server *srv, int sim_id);
/* Queues a request; *ticket identifies it for pt_server_wait.  Thread safe. */
int pt_server_submit(pt_server *srv, int sim_id, double dt_drift, double dt_kick, int64_t *ticket);
/* Waits for a request (timeout_s < 0: forever; PT_ERR_TIMEOUT when it runs
 * out) and reports its timing; each ticket can be waited for once. */
int pt_server_wait(pt_server *srv, int64_t ticket, double timeout_s, pt_request_info *info);
/* Copies a simulation's current pos, vel, acc (n x 3) and pot (n) to the given
 * buffers (host or device; NULL skips one) after its queued requests finish. */
int pt_server_read_sim(pt_server *srv, int sim_id, double *pos, double *vel, double *acc, double *pot);
/* Totals since the server started. */
int pt_server_stats(pt_server *srv, pt_server_stats_t *stats);
/* Message of the last batch that failed (empty if none); static storage in srv. */
const char *pt_server_last_error(pt_server *srv);

/* ---- introspection (copies to HOST buffers; for tests and tools) ---- */

/* info[0..4] = n, nodes, groups, max level, clusters;
 * box (5 per cluster) = origin x, y, z, S, 2^21/S. */
int pt_tree_info(pt_tree *tree, int64_t *info, double *box);

/* keys[s] = key of sorted slot s; perm[s] = original index in slot s. */
int pt_tree_keys(pt_tree *tree, uint64_t *keys, uint32_t *perm);

/* Node table in level order: ints (8 per node) = begin, count, level, leaf,
 * first_child, nchild, 0, 0; q (6 per node) = grid box min xyz, max xyz;
 * mom (10 per node) = M, centre of mass xyz, Q xx yy zz xy xz yz with
 * Q = sum m (3 d d^T - |d|^2 I) about the centre of mass. */
int pt_tree_nodes(pt_tree *tree, int64_t *ints, uint32_t *q, double *mom);

/* Groups in key order: g (8 per group) = begin, count, grid box min xyz,
 * max xyz. */
int pt_tree_groups(pt_tree *tree, int64_t *g);

/* Interaction lists of the last pt_longrange_force on this tree:
 * cell_off/pp_off (groups+1 int64), cells (node indices), pp (sorted
 * particle indices), in the order the force kernel consumed them: a group's
 * PP entries from leaves whose box lies within r_out of the group's box
 * first, then those from leaves opened for the opening angle alone (every
 * pair at least r_out apart, evaluated without the changeover test). */
int pt_tree_lists(pt_tree *tree, int64_t *cell_off, uint32_t *cells,
                  int64_t *pp_off, uint32_t *pp);

/* Version of this ABI (1). */
int pt_abi_version(void);

/* ---- orbit-dependent neighbour lists (Sec. 6.3.1, Eq. 24) ----
 *
 * Stage 1: particle i searches within r_nb,i = r_out,i + C_r |v_i| dt_L
 * (Eq. 24; r_out,i = s_i r_out with the tree's radius factors when it was
 * built mass-dependent, else r_out), and j != i is a candidate of i when
 * r_ij < max(r_nb,i, r_nb,j) -- the larger radius, as for the pair radii of
 * Eq. 12, so the relation is symmetric.  Stage 2 keeps a candidate when the
 * pericentre of the pair's two-body Kepler orbit (mu = G (m_i + m_j); from
 * the eccentricity vector, r_p = (h^2/mu) / (1 + e); the impact parameter
 * when mu = 0; r_ij when the relative velocity is 0) is below C_v R_ij.  As
 * printed, R_ij = r_nb; a pericentre never exceeds the current separation,
 * so that form keeps every candidate when C_v >= 1.  PT_ORBIT_ROUT (the
 * default reading) takes R_ij = r_out,ij = max(r_out,i, r_out,j): a
 * candidate stays when its orbit reaches the changeover region within the
 * safety factor C_v.  Every decision is made in float64, one IEEE operation
 * at a time, so the lists equal a brute-force search bit for bit. */
#define PT_ORBIT_ROUT 0         /* stage 2 with R_ij = r_out,ij */
#define PT_ORBIT_RNB 1          /* stage 2 with R_ij = r_nb,ij (as printed) */
#define PT_ORBIT_CANDIDATES 2   /* stage 1 only */

typedef struct {
    double dt;     /* dt_L, the long-range (tree) step, >= 0 */
    double C_r;    /* Eq. 24 velocity coefficient (3.0 in the paper) */
    double C_v;    /* pericentre safety factor (1.5 in the paper) */
    int mode;      /* PT_ORBIT_* */
} pt_orbit_params;

/* On a tree built by pt_tree_build(_scaled) (its positions, masses, radius
 * factors and G), with vel (n x 3 float64, input order, host or device):
 * writes the CSR lists like pt_longrange_force (nb_offsets n + 1 int64,
 * nb_idx int32 ascending within a row; NULL nb_offsets skips them), the
 * number of stored pairs to *nb_total, the number of stage-1 candidate
 * pairs (both directions) to *n_candidates, and Eq. 24's r_nb to r_nb
 * (n float64, input order) when that is not NULL; outputs host or device.
 * Too small a capacity returns PT_ERR_CAPACITY with *nb_total set.  The
 * call reuses the tree's neighbour buffers (a later pt_longrange_force
 * recomputes its own) and leaves the interaction lists untouched.
 * Returns PT_OK, PT_ERR_ARG (unbuilt tree, NULL vel/params, negative or
 * non-finite dt, C_r, C_v, unknown mode), PT_ERR_CAPACITY, PT_ERR_OOM,
 * PT_ERR_CUDA, PT_ERR_INTERNAL. */
int pt_orbit_neighbours(pt_tree *tree, const double *vel, const pt_orbit_params *params,
                        int64_t *nb_offsets, int32_t *nb_idx, int64_t nb_capacity, int64_t *nb_total,
                        int64_t *n_candidates, double *r_nb);

/* ---- tidal tensor of a binary's perturbation (Sec. 6.4.1, Eqs. 25-28) ----
 *
 * Outside its members' changeover radii, the long-range force on a binary is
 * the centre-of-mass acceleration plus a tidal correction, expanded in
 * r' = r - r_cm to first order (order 2: symmetric A_ij, 6 elements
 * xx xy xz yy yz zz) or second order (order 3: those plus the fully
 * symmetric A_ijk, 10 elements xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz, with
 * the 1/2 of the Taylor term folded into A_ijk as in Table 1):
 *     A'_i(r') = A_ij r'_j (+ A_ijk r'_j r'_k).
 * The elements are measured with zero-mass points around r_cm at distance
 * scale d_c (order 2: 4 tetrahedron corners; order 3: 8 corners; Table 1)
 * whose accelerations come from the ordinary long-range force, and are
 * solved by least squares from M T = A' (Eq. 28).
 *
 * All arrays are float64, row-major, host or device memory (host arrays are
 * staged through temporary device buffers; device arrays must be on the
 * context's device); the caller owns them.  The calls run on the context's
 * stream and return when the results are in place.  Errors: PT_ERR_ARG for
 * a NULL context or pointer with n > 0 or an order other than 2 or 3
 * (message in pt_last_error), PT_ERR_OOM, PT_ERR_CUDA.  n = 0 is a no-op. */

/* points (n x P x 3, P = 4 for order 2, 8 for order 3): measure points
 * r_cm[b] + d_c[b] * (Table 1 unit point p) of each of n binaries. */
int pt_tidal_points(pt_ctx *ctx, int order, int64_t n, const double *r_cm, const double *d_c,
                    double *points);

/* acc (n x (1 + P) x 3): per binary the long-range acceleration at r_cm
 * followed by those at its P measure points (in pt_tidal_points order).
 * T (n x E, E = 6 for order 2, 16 for order 3): the fitted elements, in the
 * order listed above. */
int pt_tidal_tensor(pt_ctx *ctx, int order, int64_t n, const double *acc, const double *d_c,
                    double *T);

/* acc_out (n_query x 3) = acc_cm[owner[q]] + the expansion of T[owner[q]] at
 * rel[q] = r_q - r_cm (n_query x 3); owner (int64) indexes the n_binaries
 * rows of T (n_binaries x E) and acc_cm (n_binaries x 3).  An owner outside
 * [0, n_binaries) gives NaN for that query and touches nothing else. */
int pt_tidal_eval(pt_ctx *ctx, int order, int64_t n_query, const int64_t *owner, const double *T,
                  int64_t n_binaries, const double *acc_cm, const double *rel, double *acc_out);

/* ---- measurement ---- */

/* Measures the float32 FMA throughput of the context's GPU: independent
 * fmaf chains, eight per thread, over 8 blocks of 256 threads per SM;
 * best of three timed launches after a warm-up (CUDA events on the
 * context's stream), in TFLOP/s (2 flops per FMA) written to *tflops.
 * About 5 ms of GPU time; allocates and frees 16 bytes.  It is the measured
 * denominator for the force kernel's fraction of peak; the paper has no
 * counterpart.  Returns PT_OK, PT_ERR_ARG, PT_ERR_OOM or PT_ERR_CUDA. */
int pt_probe_fp32_peak(pt_ctx *ctx, double *tflops);

/* ---- allocation-free entry point ---- */

/* Stable ascending sort of n 64-bit keys: keys_sorted[s] is the s-th
 * smallest key and perm[s] its index in `keys`; equal keys keep their input
 * order.  This is the same radix sort that orders the Morton keys inside
 * pt_tree_build, offered for callers that cannot allocate device memory: a
 * process whose GPU memory belongs to another allocator (a framework's
 * caching allocator or a fixed arena, where a cudaMalloc of the library's
 * own would fail or fragment it), or a loop that must never allocate.  The
 * paper has no counterpart; it is a service of this library.
 *
 * It allocates nothing.  Its scratch space is a fixed array of about
 * 4.3 MiB inside the library image, which every GPU that loads the library
 * keeps until the process exits; hence the size limit 1 <= n <= 262144
 * (2^18); larger n returns PT_ERR_ARG.
 *   keys, keys_sorted (n each, uint64) and perm (n, uint32): device memory
 *     on the calling thread's current device, owned by the caller; keys is
 *     only read.  Any other pointer kind returns PT_ERR_ARG.
 *   stream: the cudaStream_t (as void*) on which the sort is ordered; the
 *     call returns without waiting for it.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) for that device and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * this function on a device after cudaDeviceReset of that device (the kept
 * address belonged to the reset context).  All calls share the one scratch
 * array, which keeps the last call's contents (the call rewrites everything
 * it reads from it), so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.  Returns PT_OK, PT_ERR_ARG or
 * PT_ERR_CUDA (launch failure). */
int pt_sort_keys_noalloc(int64_t n, const uint64_t *keys, uint64_t *keys_sorted,
                         uint32_t *perm, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PT_H */
