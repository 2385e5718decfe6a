/*
 * tetproj.h -- C ABI of the GB300 tetrahedral-mesh CT projectors.
 *
 * The library computes the two operators every CT reconstruction algorithm
 * needs on a tetrahedral image basis (Sec. II-A of Biguri et al., "Numerically
 * robust tetrahedron-based tomographic forward and backward projectors on
 * parallel architectures"):
 *
 *   Eq. 1   A x = b + e,  a_ij = length of the intersection of ray j and tet i
 *   Eq. 2   forward projection   b_j = sum_i a_ij mu_i
 *   Eq. 3   backprojection       x_i = sum_j a_ij y_j     (the exact adjoint A^T)
 *
 * A is never stored: each call walks every ray through the mesh, tet to tet
 * across shared faces (Alg. 2), starting from the boundary face where the ray
 * enters (Sec. II-E, here found through a bounding-volume hierarchy over the
 * boundary faces).  Exit faces are decided by exact-sign orientation
 * predicates with a symbolic tie-break, so no ray can leak or loop.
 *
 * Conventions shared by all calls
 * -------------------------------
 * - A ray is the half-line X(t) = S + t (P - S), t >= 0, from a source S through
 *   a point P (a detector pixel centre).  S may lie anywhere (inside the mesh
 *   too: only the part of the line with t >= 0 is integrated).
 * - Cone-beam geometry (circular orbit about z, flat detector): for angle theta
 *   S = (dso cos, dso sin, 0), detector centre C = S - dsd (cos, sin, 0),
 *   u axis U = (-sin, cos, 0), v axis V = (0, 0, 1), pixel centre
 *   P = C + u U + v V with u = (iu - (nu-1)/2) du, v = (iv - (nv-1)/2) dv.
 *   Ray index j = (a * nv + iv) * nu + iu.
 * - Layouts: mu / mu_out are [nt][C] in the user's tet order; projections are
 *   [nangles][nv][nu][C]; explicit rays take src/dst as [n][3] FP64.
 * - Element type: float for TETPROJ_FILTERED, double for TETPROJ_PLAIN_FP64.
 *   C (channels, several attenuation maps sharing one traversal) is 1 or 4.
 * - Every data pointer passed to forward/backward/trace is a DEVICE pointer
 *   owned by the caller.  Host pointers appear only in the *_create calls and
 *   in the *_host helpers.  `stream` is a cudaStream_t (NULL = legacy stream).
 * - Compute calls are asynchronous and ordered on `stream`; they never
 *   synchronise and never allocate, except that the first forward/backward on a
 *   mesh with a given (precision, channels) allocates the mesh's workspace
 *   (tetproj_mesh_reserve does that up front, e.g. before CUDA-graph capture).
 *   Argument errors are returned immediately.  Errors met on the device (a walk
 *   that exceeds max_steps) are recorded in the mesh's counters and reported
 *   by tetproj_mesh_stats_read; the affected outputs are NaN.
 * - Calls on the same mesh share its workspace and counters: issue them on one
 *   stream (or order them with events).
 */
#ifndef TETPROJ_H
#define TETPROJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tetproj_status;

#define TETPROJ_OK 0
#define TETPROJ_ERR_ARG 1             /* invalid argument (NULL, size, option)      */
#define TETPROJ_ERR_INDEX 2           /* vertex index out of range or repeated        */
#define TETPROJ_ERR_DEGENERATE_TET 3  /* zero-volume tet (exact orientation = 0)      */
#define TETPROJ_ERR_NONMANIFOLD 4     /* face shared by >2 tets, overlapping tets     */
#define TETPROJ_ERR_NONCONVEX 5       /* boundary surface not convex (Sec. II-D)      */
#define TETPROJ_ERR_CUDA 6            /* a CUDA runtime call failed                   */
#define TETPROJ_ERR_OOM 7             /* device or host allocation failed             */
#define TETPROJ_ERR_RAY_LIMIT 8       /* a walk exceeded max_steps (device-side)      */
#define TETPROJ_ERR_TIMEOUT 9         /* a bounded device wait gave up (device-side)  */
#define TETPROJ_ERR_SOURCE_INSIDE 10  /* reserved (sources inside the mesh are supported) */
#define TETPROJ_ERR_TOO_LARGE 11      /* mesh or problem exceeds a documented limit   */

/* precision modes */
#define TETPROJ_FILTERED 0   /* FP32 data; FP32 predicates with a forward error bound,
                                FP64 / exact / symbolic fallback; Kahan FP32 sums     */
#define TETPROJ_PLAIN_FP64 1 /* FP64 data, predicates (FP64 filter + exact), sums, atomics */

/* pixel order inside a ray tile */
#define TETPROJ_ORDER_ROW 0
#define TETPROJ_ORDER_MORTON 1

/* backprojection scatter */
#define TETPROJ_SCATTER_ATOMIC 0  /* one atomic add per segment                     */
#define TETPROJ_SCATTER_WARP 1    /* lanes of a warp on the same tet merge first     */
#define TETPROJ_SCATTER_SORT 2    /* segment sort-and-reduce: deterministic (see
                                     tetproj_backward); filtered path, cone rays   */

/* options.flags */
#define TETPROJ_FLAG_RSTAR_ENTRY 1 /* entry search through an R*-tree of the boundary
                                      faces (the paper's structure, Sec. II-E)
                                      instead of the binary BVH: filtered forward
                                      (C = 1) and tetproj_entry only; the tree is
                                      built on first use (synchronous)          */
#define TETPROJ_FLAG_ACC64 2       /* filtered backprojection with atomic or
                                      warp-aggregated scatter: add the FP32
                                      segment contributions into an FP64
                                      accumulator (red.global.add.f64; with
                                      _SCATTER_WARP, lanes at one tet are summed
                                      in FP64 first, one reduction per tet) and
                                      round once: ~1e-7 for any number of
                                      segments per tet.  Default for C = 1.    */
#define TETPROJ_FLAG_ACC32 4       /* the same into an FP32 accumulator (faster for
                                      C = 4: one 16-byte red per segment instead
                                      of four 8-byte ones; FP32 sums drift like
                                      sqrt(segments per tet) * 2^-24).  With
                                      neither ACC flag, C = 4 uses FP32 too, but
                                      two-level on dense meshes (nt * C <= 2^20
                                      and >= 64 rays per element): the FP32
                                      accumulator is merged into an FP64 one
                                      after every chunk of at most
                                      max(2^18, 8192 nt / s) rays, s = 1.5
                                      (nt / 6)^(1/3) + 1 (segments per ray
                                      estimate).  ACC32 keeps it
                                      single-level.  At most one ACC flag.     */

typedef struct tetproj_mesh tetproj_mesh;
typedef struct tetproj_geometry tetproj_geometry;

typedef struct tetproj_options {
    int32_t precision; /* TETPROJ_FILTERED (default) or TETPROJ_PLAIN_FP64            */
    int32_t channels;  /* C: 1 (default) or 4                                          */
    int32_t tile_u;    /* ray tile width in pixels: 1..32, power of two (default 16)   */
    int32_t tile_v;    /* ray tile height: tile_u*tile_v in {32,64,128,256} (def. 8)   */
    int32_t order;     /* TETPROJ_ORDER_MORTON (default) or TETPROJ_ORDER_ROW          */
    int32_t scatter;   /* TETPROJ_SCATTER_ATOMIC (default), _WARP or _SORT             */
    int32_t max_steps; /* walk step limit per ray; 0 = 64 + 16*ceil(nt^(1/3))          */
    int32_t flags;     /* 0 or an or of TETPROJ_FLAG_* (RSTAR_ENTRY, ACC64 | ACC32)   */
} tetproj_options;

typedef struct tetproj_stats {
    int64_t rays;        /* rays launched                                              */
    int64_t hits;        /* rays that entered the mesh                                 */
    int64_t segments;    /* tet visits (walk steps), zero-length visits included       */
    int64_t fp64_filter; /* edge predicates the FP32 filter could not decide           */
    int64_t exact;       /* ... that the FP64 filter could not decide either           */
    int64_t sos;         /* ... that were exactly zero (symbolic tie-break used)        */
    int64_t bvh_nodes;   /* BVH boxes tested by entry searches                         */
    int64_t bvh_faces;   /* boundary faces tested by entry searches                    */
    int64_t deferred;    /* rays the fast FP32 walk handed to the robust resume walk   */
    int32_t error;       /* first device-side error code, 0 if none                    */
    int32_t error_count; /* rays that hit a device-side error                          */
    int64_t grazing;     /* crossings at a grazing angle placed again from FP64 records */
} tetproj_stats;

typedef struct tetproj_mesh_info {
    int64_t nt, nv;          /* tets, vertices                                         */
    int64_t nboundary;       /* boundary faces                                         */
    int64_t nbvh_nodes;      /* BVH nodes                                              */
    int64_t nflipped;        /* input tets that were negatively oriented (re-ordered)  */
    int64_t device_bytes;    /* device memory held by the mesh (records, BVH, workspace) */
    double bbox[6];          /* xmin, ymin, zmin, xmax, ymax, zmax                     */
} tetproj_mesh_info;

/* Fills *opt with the defaults listed above. */
void tetproj_default_options(tetproj_options *opt);

/* Static description of a status code (never NULL). */
const char *tetproj_status_string(tetproj_status s);

/* ---------------------------------------------------------------- meshes --
 * tetproj_mesh_create: builds the device mesh from HOST arrays (Sec. II-B, the
 * element/neighbour graph, and Sec. II-E, the boundary list and search tree).
 *   vertices: [nv][3] FP64;  tets: [nt][4] int32 vertex indices (any orientation).
 * Copies its inputs; the caller may free them on return.  Validates the mesh
 * (indices, zero-volume tets, faces shared by more than two tets or by two tets
 * on the same side, convexity of the boundary), re-orders each tet's vertices
 * to positive orientation, builds face adjacency, renumbers tets along a 3-D
 * Hilbert curve of their centroids, builds the boundary-face BVH and uploads
 * everything with synchronous copies on the current device.  Limits:
 * nt < 2^29, nv < 2^31, |coordinates| < 1e9.  On error *out is NULL. */
tetproj_status tetproj_mesh_create(const double *vertices, int64_t nv, const int32_t *tets,
                                   int64_t nt, tetproj_mesh **out);

/* Frees the mesh and its device memory (synchronises the device first). */
tetproj_status tetproj_mesh_destroy(tetproj_mesh *mesh);

tetproj_status tetproj_mesh_get_info(const tetproj_mesh *mesh, tetproj_mesh_info *out);

/* Allocates the mesh's workspace for (precision, channels) now instead of on
 * the first compute call: operand/accumulator buffers and the deferral queue,
 * for the filtered path also the FP64 accumulator its backprojection uses by
 * default at C = 1 (and at C = 4 when nt * 4 <= 2^20).  The queue holds one
 * launch chunk, min(rays, 2^24), at 80 B per ray (1.25 GB at 2^24).  Calls of
 * more than 2^24 rays add a second queue and a stream on first use to overlap
 * their chunks; under CUDA-graph capture they run without them rather than
 * allocate.  Synchronous. */
tetproj_status tetproj_mesh_reserve(tetproj_mesh *mesh, int32_t precision, int32_t channels);

/* Host-only topology of a mesh, in the user's tet order (no device needed):
 * adj_out [nt][4]: tet across the face opposite local vertex k of the INPUT
 * tet, or -1 on the boundary; *nboundary_out: boundary face count;
 * *nflipped_out: negatively oriented input tets.  Same validation as create. */
tetproj_status tetproj_mesh_topology_host(const double *vertices, int64_t nv,
                                          const int32_t *tets, int64_t nt, int32_t *adj_out,
                                          int64_t *nboundary_out, int64_t *nflipped_out);

/* Zeroes / reads the mesh's device counters (read synchronises `stream`). */
tetproj_status tetproj_mesh_stats_reset(tetproj_mesh *mesh, void *stream);
tetproj_status tetproj_mesh_stats_read(tetproj_mesh *mesh, void *stream, tetproj_stats *out);

/* -------------------------------------------------------------- geometry --
 * Circular cone-beam scan (Alg. 2 launches one ray per detector pixel; the
 * paper's experiments use equidistant angles over a circular trajectory).
 *   dso: source to rotation axis; dsd: source to detector (> dso);
 *   nu, nv: detector pixels; du, dv: pixel pitch; angles: HOST [nangles] rad.
 * Per-angle frames are computed on the host in FP64 and uploaded. */
tetproj_status tetproj_geometry_create(double dso, double dsd, int32_t nu, int32_t nv, double du,
                                       double dv, const double *angles, int32_t nangles,
                                       tetproj_geometry **out);
tetproj_status tetproj_geometry_destroy(tetproj_geometry *geo);

/* Writes the endpoints (S, P) of the rays with the given indices (device
 * int64 [n]; NULL = rays 0..n-1) into device src/dst [n][3] FP64. */
tetproj_status tetproj_geometry_rays(const tetproj_geometry *geo, const int64_t *ray_idx,
                                     int64_t n, double *src, double *dst, void *stream);

/* ------------------------------------------------------------- operators --
 * tetproj_forward (Eq. 2): proj[a][iv][iu][c] = sum_i a_ij mu[i][c].
 *   mu: device [nt][C]; proj: device [nangles][nv][nu][C] (overwritten).
 * tetproj_backward (Eq. 3): mu_out[i][c] = sum_j a_ij proj[j][c] (overwritten).
 * opt may be NULL (defaults).  Both are exact adjoints of each other up to
 * floating-point rounding.
 * Backprojection scatter (Sec. II-F adds with atomics): _ATOMIC and _WARP add
 * each segment's length x y into its tet atomically, in an order the hardware
 * picks.  _SORT (filtered path only) writes the segments (tet, length x y) of
 * a chunk of rays to a buffer at positions fixed by the rays' segment counts,
 * sorts them stably by tet and sums each tet's run in that order, so the
 * result is bit-reproducible.  Its first call for a (mesh, geometry, tile
 * shape, ordering, C) builds a segment plan (a counting walk; synchronous;
 * 8 B per ray + 16 B per tile block), reused while the mesh's last plan
 * matches; sort buffers for chunks of 2^29 segments at C = 1 (8.6 GB) or 2^27
 * at C = 4 (6.4 GB) are allocated on first use.  Later calls are
 * asynchronous and allocate nothing.
 * Errors of the counting walk are returned by the call that builds the plan. */
tetproj_status tetproj_forward(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                               const void *mu, void *proj, const tetproj_options *opt,
                               void *stream);
tetproj_status tetproj_backward(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                                const void *proj, void *mu_out, const tetproj_options *opt,
                                void *stream);

/* tetproj_backward without any allocation.  It computes the same x = A^T y as
 * tetproj_backward (same arguments, layouts, options and accumulator: FP64 at
 * C = 1 on the filtered path unless TETPROJ_FLAG_ACC32, two-level FP32 -> FP64
 * for dense problems at C = 4, FP32 otherwise, FP64 on the plain path), for
 * callers that cannot call cudaMalloc when they backproject: code whose device
 * memory is wholly owned by another allocator (e.g. a framework's caching pool
 * that has reserved the device), or a latency-critical loop that must not pay
 * cudaMalloc's implicit synchronisation.  The paper has no counterpart; this
 * is a library facility.  TETPROJ_SCATTER_SORT is not offered
 * (TETPROJ_ERR_ARG): its buffers grow with the number of segments.
 * Its scratch (accumulator and deferral queue) is a fixed device array inside
 * the library, present on every GPU that loads it until the process exits:
 *   - limit: the accumulator must fit TETPROJ_NOALLOC_ACC_BYTES, else
 *     TETPROJ_ERR_TOO_LARGE: nt * C * 8 bytes with an FP64 accumulator (the
 *     filtered C = 1 default: up to 4,194,304 tets; plain FP64), nt * C * 4
 *     with FP32 (C = 4 sparse problems, TETPROJ_FLAG_ACC32), and 12 nt C for
 *     the dense two-level case (always fits: dense means nt C <= 2^20);
 *   - the first call on a device (and the first after that device's context
 *     was destroyed and created again) looks up the array's device address
 *     (no allocation); make that first call before any stream capture;
 *   - all calls share the array and it keeps the last call's contents (each
 *     call clears what must start at zero); calls that overlap on the GPU
 *     (unordered streams) race on it. */
#define TETPROJ_NOALLOC_ACC_BYTES (32 * 1024 * 1024)
tetproj_status tetproj_backward_noalloc(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                                        const void *proj, void *mu_out,
                                        const tetproj_options *opt, void *stream);

/* The same operators for explicit rays src[j] -> dst[j] (device [n][3] FP64):
 * out[j][c] = sum_i a_ij mu[i][c];  mu_out[i][c] = sum_j a_ij y[j][c]. */
tetproj_status tetproj_forward_rays(const tetproj_mesh *mesh, const double *src,
                                    const double *dst, int64_t nrays, const void *mu, void *out,
                                    const tetproj_options *opt, void *stream);
tetproj_status tetproj_backward_rays(const tetproj_mesh *mesh, const double *src,
                                     const double *dst, int64_t nrays, const void *y,
                                     void *mu_out, const tetproj_options *opt, void *stream);

/* Row j of A for explicit rays: the tets visited, in order, with their chord
 * lengths a_ij (zero-length visits at edges/vertices included).
 *   out_tet: device int32 [n][max_visits] user tet ids; out_len: device FP64
 *   [n][max_visits]; out_count: device int32 [n] visits (may exceed max_visits;
 *   entries past max_visits are not written).  opt->precision selects the walk. */
tetproj_status tetproj_trace_rays(const tetproj_mesh *mesh, const double *src, const double *dst,
                                  int64_t nrays, int32_t max_visits, int32_t *out_tet,
                                  double *out_len, int32_t *out_count,
                                  const tetproj_options *opt, void *stream);

/* --------------------------------------------------------------- batches --
 * Many independent problems (mesh, geometry) of uneven size projected in one
 * persistent work-queue launch per round: warps take (problem, angle, tile,
 * 32-ray slice) items from an atomic counter, so large and small problems
 * share the GPU without per-problem launch tails (the paper splits projections across GPUs,
 * Sec. II-F; here many problems share one GPU).  Filtered FP32 path only.
 *   meshes, geos: HOST arrays of n handles (a mesh may appear several times);
 *   tiles: HOST [n][4] = (tile_u, tile_v, order, scatter) per problem, or NULL
 *          for the defaults; each as in the options struct (powers of two,
 *          32..256 rays per tile); problems may use different tiles;
 *   channels: C = 1 or 4 for every problem.
 * The batch owns per-problem workspace and one deferral queue of
 * min(total rays, 2^25) entries at 80 B (2.5 GB at 2^25; a second one when
 * there are several rounds), allocated here; it keeps pointers into the
 * meshes and geometries, which must outlive
 * it.  Backprojections add into FP64 accumulators at C = 1 (with each problem's
 * atomic or warp-aggregated scatter) and into FP32 ones at C = 4, two-level
 * for dense problems (as TETPROJ_FLAG_ACC32 describes; merged after every
 * round).  Rays are processed in rounds of at most 2^25 rays; backprojection
 * rounds are cut further inside dense problems (at most max(2^18,
 * 8192 nt / s) of their rays per round, as above).
 * Errors: TETPROJ_ERR_ARG (null handle, n < 1, bad channels or tiles),
 * TETPROJ_ERR_TOO_LARGE (2^40 work items or more), CUDA
 * errors of the allocations; *out is NULL on error. */
typedef struct tetproj_batch tetproj_batch;
tetproj_status tetproj_batch_create(const tetproj_mesh *const *meshes,
                                    const tetproj_geometry *const *geos, const int32_t *tiles,
                                    int32_t n, int32_t channels, tetproj_batch **out);
/* Binds the operands: HOST arrays of n DEVICE pointers (float, layouts as in
 * tetproj_forward/backward).  mu/proj are used by tetproj_batch_forward, y/mu_out
 * by tetproj_batch_backward; the pair not used may be NULL.  Synchronous
 * (uploads the per-problem tables). */
tetproj_status tetproj_batch_bind(tetproj_batch *b, const void *const *mu, void *const *proj,
                                  const void *const *y, void *const *mu_out);
/* proj[k] = A_k mu[k] and mu_out[k] = A_k^T y[k] for every problem; async on
 * `stream`, no allocation and no host synchronisation: the sequence can be
 * captured in a CUDA graph (the graph then replays with the bound buffers). */
tetproj_status tetproj_batch_forward(tetproj_batch *b, void *stream);
tetproj_status tetproj_batch_backward(tetproj_batch *b, void *stream);
tetproj_status tetproj_batch_destroy(tetproj_batch *b);
/* The persistent launch hands work to the warps of a CTA through two waits on
 * shared-memory words that other warps of the CTA write (this build's work
 * queue, not the paper's).  Each wait gives up after a bounded number of polls
 * (2^22, tens of milliseconds): the call then completes with incomplete
 * results and the mesh statistics report TETPROJ_ERR_TIMEOUT, and the context
 * stays usable.  This sets the bound for later calls of this batch (a CUDA
 * graph keeps the value it was captured with): max_polls > 0 polls, 0 the
 * default.  never_satisfied != 0 makes every wait wait for a value no warp
 * writes, so each runs out after max_polls polls: a test of the timeout path,
 * not for production use.  Errors: TETPROJ_ERR_ARG (null batch, max_polls < 0). */
tetproj_status tetproj_batch_set_wait(tetproj_batch *b, int32_t max_polls,
                                      int32_t never_satisfied);

/* ------------------------------------------------- the paper's own walk --
 * Alg. 1 and 2 as printed (Sec. II-C..E): Moller-Trumbore ray-triangle tests
 * with a safety margin eps = 1e-9 multiplied by 10 until two faces of the
 * current tet are hit; the walk leaves through the face of the larger hit
 * parameter.  A COMPARISON mode for the paper's floating-point experiment
 * (Sec. III-C): FP32 (TETPROJ_FILTERED selects single precision here) or FP64
 * (TETPROJ_PLAIN_FP64) arithmetic throughout, no exact predicates.  Forward
 * only, C = 1, tiles of at most 128 rays.  status (device int8 [nrays], or
 * NULL): 0 = walk completed (or missed the mesh), 1 = halted (eps reached
 * 1e-2 without two intersections: a missed exit), 2 = more than max_steps
 * tets (looping).  Halted and looping rays return their partial sums.
 * Readings of what the paper leaves open are listed in kernels.cu. */
tetproj_status tetproj_forward_mt(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                                  const void *mu, void *proj, int8_t *status,
                                  const tetproj_options *opt, void *stream);
tetproj_status tetproj_forward_rays_mt(const tetproj_mesh *mesh, const double *src,
                                       const double *dst, int64_t nrays, const void *mu,
                                       void *out, int8_t *status, const tetproj_options *opt,
                                       void *stream);

/* ---------------------------------------------------------- entry search --
 * entry_tet[ray] = user id of the first tet each cone ray enters (-1: the ray
 * misses the mesh): the entry search alone (Sec. II-E), filtered precision,
 * through the BVH or, with TETPROJ_FLAG_RSTAR_ENTRY, the R*-tree.  entry_tet:
 * device int32 [nangles][nv][nu]. */
tetproj_status tetproj_entry(const tetproj_mesh *mesh, const tetproj_geometry *geo,
                             int32_t *entry_tet, const tetproj_options *opt, void *stream);

typedef struct tetproj_rstar_info {
    int64_t nodes, leaves, entries; /* entries: boundary faces listed in leaves      */
    int32_t depth;                  /* levels, root to leaves                        */
    int32_t min_fill, max_fill;     /* entries per non-root node                     */
    int32_t ok;                     /* 1: fills within [4, 10], leaves at one depth,
                                       boxes nested, every face in exactly one leaf */
} tetproj_rstar_info;
/* Builds the mesh's boundary-face R*-tree on the host (no device needed) and
 * checks its invariants; HOST inputs as tetproj_mesh_create. */
tetproj_status tetproj_rstar_build_host(const double *vertices, int64_t nv, const int32_t *tets,
                                        int64_t nt, tetproj_rstar_info *out);

/* ------------------------------------------------------------ predicates --
 * Sign of the side product det[P - S, p - S, q - S] of the line S->P and the
 * edge p->q (the test behind each of the four triangle tests of Sec. II-C),
 * evaluated by the library's cascade: FP32 with a forward error bound, then
 * FP64 with an error bound, then exact expansion arithmetic, then the
 * symbolic perturbation of the line (S + (e, e^2, e^4), P + (e^8, e^16, e^32),
 * e -> 0+) when the exact value is zero.  sign[k] in {-1, +1} (0 only if
 * p == q); stage[k]: 0 FP32, 1 FP64, 2 exact, 3 symbolic.
 * _host: host arrays, runs on the CPU.  _device: device arrays, on `stream`. */
tetproj_status tetproj_side_host(const double *S, const double *P, const double *p,
                                 const double *q, int64_t n, int8_t *sign, int8_t *stage);
tetproj_status tetproj_side_device(const double *S, const double *P, const double *p,
                                   const double *q, int64_t n, int8_t *sign, int8_t *stage,
                                   void *stream);

/* Library version (major*10000 + minor*100 + patch). */
int32_t tetproj_version(void);

/* Number of CUDA kernels this library has launched in this process, counted
 * on the host at each launch (for benchmarks; no counterpart in the paper).
 * Kernels replayed from a captured CUDA graph are counted once, at capture. */
int64_t tetproj_launch_count(void);

/* FP64 FMA throughput probe (for benchmarks; no counterpart in the paper).
 * Launches 8 x SM-count CTAs of 256 threads on `stream`, each thread running
 * 8 independent chains of `iters` FP64 FMAs; *flops receives the
 * floating-point operations launched (2 per FMA), so flops / (event-timed
 * duration) is the device's FP64 FMA rate, the roofline of the plain FP64
 * walk.  sink: device buffer of 8 x SM-count doubles (never written in
 * practice).  Errors: TETPROJ_ERR_ARG (iters < 1, NULL pointers), CUDA. */
tetproj_status tetproj_fma64_probe(int64_t iters, double *sink, double *flops, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TETPROJ_H */
