/*
 * pndf.h - C ABI of the GB300 P-NDF library (libpndf.so).
 *
 * Position-normal manifold P-NDF evaluation (Wu, Luan, Hasan, Ramamoorthi,
 * "Position-Normal Manifold for Efficient Glint Rendering on High-Resolution
 * Normal Maps", Sec. 4) and the analytic projected-area integral (Sec. 4.3,
 * App. B).  Every function here is host-callable C; no C++ or framework type
 * crosses this boundary.  All compute runs in CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point
 *   - Texel u = (i, j) of an N x N normal map sits at element j*N + i
 *     (row-major, i along x).  Its value is the projected-hemisphere normal
 *     n = (s, t) (Sec. 3, Eq. 2).  Positions are unnormalised texel units
 *     (Tab. 1).
 *   - Quad (i, j), 0 <= i, j <= N-2, is split along the u1-u2 diagonal into
 *     a lower triangle (u0, u1, u2) and an upper triangle (u3, u2, u1)
 *     (Eq. 3).  Triangle id = 2 * (j*(N-1) + i) + (0 lower | 1 upper).
 *   - The footprint kernel k_r is the Gaussian exp(-q/2) / (2 pi sqrt(det S))
 *     with q = d^T S^-1 d, cut to zero where q > 16 (the 4-sigma ellipse),
 *     not renormalised.  The map is not periodic.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream.  Argument errors are
 *     returned synchronously; device-side errors (invalid query, capacity)
 *     set a per-device status word read by pndf_device_status().
 *   - Buffers named *_dev are device pointers owned by the caller; the
 *     library never frees them and reads/writes them only within the call's
 *     stream order.  Hierarchies are library-owned device memory.
 *   - Thread safety: distinct streams may call concurrently.  A hierarchy is
 *     immutable after its build completes, so concurrent evaluations on it
 *     are safe; it must not be freed while work on it is in flight.
 */
#ifndef PNDF_H
#define PNDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pndf_hierarchy pndf_hierarchy;

typedef enum pndf_status {
    PNDF_OK = 0,
    PNDF_ERR_INVALID_ARG = 1,  /* bad pointer, size, format or parameter            */
    PNDF_ERR_OOM = 2,          /* device allocation failed                          */
    PNDF_ERR_CUDA = 3,         /* a CUDA runtime call failed                        */
    PNDF_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out                */
    PNDF_ERR_CAPACITY = 5,     /* a fixed-size device buffer would overflow         */
    PNDF_ERR_UNSUPPORTED = 6,  /* valid request this build does not implement       */
    PNDF_ERR_DEVICE = 7        /* pndf_device_status: a kernel recorded an error     */
} pndf_status;

typedef enum pndf_texel_fmt {
    PNDF_TEXEL_F32X2 = 0,      /* float  (s, t) pairs, 8 bytes per texel            */
    PNDF_TEXEL_F16X2 = 1       /* binary16 (s, t) pairs, 4 bytes per texel           */
} pndf_texel_fmt;

typedef enum pndf_bounds_fmt {
    PNDF_BOUNDS_F32 = 0,           /* exact float32 min/max per node (16 B)         */
    PNDF_BOUNDS_F16_OUTWARD = 1    /* binary16 min rounded down, max rounded up (8 B) */
} pndf_bounds_fmt;

typedef struct pndf_build_params {
    int32_t n;           /* texels per side, 2 <= n <= 16384                      */
    int32_t texel_fmt;   /* pndf_texel_fmt                                        */
    int32_t bounds_fmt;  /* pndf_bounds_fmt                                       */
    int32_t leaf_level;  /* 0 = default (2): stored bottom level, 2^l x 2^l quads */
    int32_t clusters;    /* 1 = also build the cluster hierarchy (Sec. 4.2, Eq.   */
                         /* 7-8) used by pndf_eval_config.tau; 0 = none           */
} pndf_build_params;

/* One P-NDF query, 32 bytes: footprint centre x = (x, y) in texels, the 2x2
 * footprint covariance S = [[sxx, sxy], [sxy, syy]] in texel^2 (must be
 * positive definite), and the query normal m = (ms, mt) (Eq. 2). */
typedef struct pndf_query {
    float x, y, sxx, sxy, syy, ms, mt, pad;
} pndf_query;

/* Optional per-query counters (40 bytes), written when stats_dev != NULL. */
typedef struct pndf_query_stats {
    uint32_t nodes;        /* hierarchy nodes tested                                 */
    uint32_t leaf_blocks;  /* leaf blocks whose triangles were tested                */
    uint32_t tri_tests;    /* triangles tested against m                             */
    uint32_t hits;         /* contributing hits (m inside, q <= 16)                  */
    uint32_t hit_hash;     /* sum mod 2^32 of MurmurHash3-fmix32(triangle id) over hits */
    uint32_t fp64_tris;    /* triangles evaluated in FP64 (normal area < 1e-10)      */
    uint32_t degenerate;   /* zero-area normal triangles met inside their bbox       */
    uint32_t quads;        /* per-quad (level 0) boxes tested                        */
    uint32_t cluster_checks; /* nodes whose cluster residual was compared with the cut */
    uint32_t clusters;     /* cluster nodes whose two triangles were tested          */
} pndf_query_stats;

/* Per-query flag bits written to flags_out_dev. */
#define PNDF_QF_FP64 1u       /* a triangle of normal-space area < 1e-10 was hit-tested in FP64 */
#define PNDF_QF_INVALID 4u    /* covariance not positive definite: D = NaN                       */
#define PNDF_QF_OVERFLOW 8u   /* traversal stack overflow: D incomplete (never expected)          */

typedef enum pndf_eval_mode {
    PNDF_MODE_HIERARCHY = 0,  /* min/max bound-pyramid traversal (Sec. 4.2)          */
    PNDF_MODE_FLAT = 1        /* every leaf block in the footprint box, no pruning   */
} pndf_eval_mode;

typedef enum pndf_sort_mode {
    PNDF_SORT_NONE = 0,         /* caller order                                       */
    PNDF_SORT_LEVEL_TILE = 1,   /* entry level (largest first), then centre tile (default) */
    PNDF_SORT_LEVEL_NORMAL = 2, /* entry level, then query-normal bin                    */
    PNDF_SORT_LEVEL_TILE_NORMAL = 3, /* entry level, centre tile, then normal bin          */
    PNDF_SORT_LEVEL_NORMAL_TILE = 4  /* entry level, normal bin, then centre tile          */
} pndf_sort_mode;
#define PNDF_SORT_DEFAULT PNDF_SORT_LEVEL_TILE

/* Footprint kernel k_r(d), d = u - x, q = d^T S^-1 d (Eq. 2; the Gaussian of
 * Sec. 5 and the disk and box filters of the kernel ablation, whose (3
 * sigma)^2 footprints the paper pairs with the Gaussian's (6 sigma)^2):
 *   GAUSS exp(-q/2) / (2 pi sqrt(det S)) where q <= 16 (4 sigma), else 0;
 *   DISK  1 / (2.25 pi sqrt(det S)) where q <= 1.5^2, else 0;
 *   BOX   1 / (9 sqrt(det S)) where |L^-1 d|_inf <= 1.5, S = L L^T (Cholesky),
 *         else 0 (for S = sigma^2 I, the square of side 3 sigma). */
typedef enum pndf_kernel {
    PNDF_KERNEL_GAUSS = 0,
    PNDF_KERNEL_DISK = 1,
    PNDF_KERNEL_BOX = 2
} pndf_kernel;

typedef struct pndf_eval_config {
    int32_t mode;           /* pndf_eval_mode                                         */
    int32_t sort;           /* query order before traversal (pndf_sort_mode)          */
    int32_t warps_per_cta;  /* 0 = library default                                   */
    int32_t ctas_per_sm;    /* 0 = as many as fit                                    */
    float tau;              /* cluster cut (Sec. 4.2): a node whose residual e <=      */
                            /* r_x r_y tau is evaluated as its two cluster triangles;  */
                            /* 0 = exact (no cluster).  Needs a hierarchy built with   */
                            /* clusters = 1, else UNSUPPORTED.  Hierarchy mode only.   */
    int32_t kernel;         /* footprint kernel (pndf_kernel)                          */
    float jac_eps;          /* Jacobian clamp of Eq. 6: 0 = exact; else (>= 1e-9, e.g.  */
                            /* 1e-6) a fine triangle with |cross| < jac_eps counts as  */
                            /* an equilateral one of Jacobian jac_eps centred at its   */
                            /* normal centroid.  Gaussian kernel, hierarchy mode, no   */
                            /* cluster cut (else UNSUPPORTED).                         */
    int32_t split;          /* 0 = library default: a footprint whose support box is   */
                            /* much larger than the batch's average share per warp is  */
                            /* divided into tiles of pyramid nodes evaluated by        */
                            /* several warps (hierarchy mode without the cluster cut);  */
                            /* -1 = one warp per query.  The result is the same bits   */
                            /* either way (each query's sum is exact); only the node   */
                            /* count in the stats differs.                             */
    void *ev_begin;         /* optional cudaEvent_t recorded on the stream just before */
    void *ev_end;           /* and just after the traversal kernel (NULL = none)       */
} pndf_eval_config;

/*
 * Build the min/max normal-bound pyramid of a normal map (Sec. 4.2, Fig. 5a).
 * A node at level l covers 2^l x 2^l quads; it stores the bounding box of the
 * normals of all texels of its quads, so the normal triangles of every quad
 * below it lie inside.  Levels leaf_level..L are stored (2^L >= N-1), each
 * in Morton order so the four children of a node are contiguous, plus level
 * 0 (one box per quad, Morton order, so a leaf block's 16 quads are
 * contiguous) and beside it one capsule per quad (8 bytes: the segment
 * between the quad's two farthest normals and a radius holding all four, a
 * tighter filter than the box for the long slivers of quads that straddle
 * two normal regions); nodes without quads hold an empty box.  The texels are copied into the
 * hierarchy (the caller may free texels_dev once the stream reaches the end
 * of this call's work).  On success *out owns device memory until
 * pndf_free_hierarchy().
 *   texels_dev: N*N texels in params->texel_fmt, row-major, in device memory
 *     of the current device or in page-locked host memory (cudaHostAlloc /
 *     cudaHostRegister; the build kernel then reads the map straight over the
 *     host link, with no staging copy).  Other pointers (pageable host
 *     memory, another device's memory) are rejected with INVALID_ARG before
 *     any work is queued.
 * With params->clusters = 1 the cluster hierarchy of Sec. 4.2 is built too:
 * every node of level >= 2 whose quads all lie inside the map gets the four
 * corner normals of a two-triangle cluster (split like a quad) minimising
 * the Jacobian-weighted L2 error of Eq. 7 (|det J| clamped at 1e-6 as in
 * Eq. 6), solved in FP64, and its residual e = sqrt of the minimum (the
 * 2-norm of Eq. 8, units texel^2).  Each node box is widened to hold its own
 * cluster corners and its children's boxes, so pruning never hides a cluster
 * triangle; 36 more bytes per node of level >= 2.
 * Errors: INVALID_ARG (null pointers, N out of range, unknown formats,
 *         clusters not 0 or 1), UNSUPPORTED (leaf_level), OOM, CUDA.
 */
pndf_status pndf_build_hierarchy(const void *texels_dev, const pndf_build_params *params,
                                 void *stream, pndf_hierarchy **out);

/* Rebuild h in place from new texels of the same size and format (the map
 * changed): copies the texels and recomputes every pyramid level on stream,
 * with no allocation.  texels_dev as for pndf_build_hierarchy (device memory
 * or page-locked host memory).  Work already queued on h must be on the same
 * stream or complete.  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_update_hierarchy(pndf_hierarchy *h, const void *texels_dev, void *stream);

/* Release a hierarchy (synchronises its device memory release with the
 * device; safe on NULL). */
void pndf_free_hierarchy(pndf_hierarchy *h);

/* Device bytes held by a hierarchy (texel copy + pyramid + per-quad
 * capsules + status word, and the cluster records when built). */
size_t pndf_hierarchy_bytes(const pndf_hierarchy *h);

/* Per-sample flags of pndf_sample_normals. */
#define PNDF_SF_INVALID 1u    /* covariance not positive definite: m = 0                        */
#define PNDF_SF_OUTSIDE 2u    /* the sampled uv point lies outside the map: m = 0               */

/*
 * P-NDF sampling (Sec. 3, Eq. 6): one normal per record of q_dev (its x and S
 * are used), drawn by sampling the footprint kernel u ~ k_r(u - x) and
 * querying m = n(u) (Eq. 3); with jac_eps > 0 a fine triangle whose |cross|
 * is below jac_eps stands for its equilateral replacement (as in
 * pndf_eval_config.jac_eps), so the sampled normals have density D (clamped
 * alike) over the kernel mass.  u is the inverse CDF of the caller's two
 * uniforms per sample in the whitened frame v (u = x + L v, S = L L^T):
 * Gaussian (cut at 4 sigma) |v|^2 = -2 ln(1 - U1 (1 - e^-8)), angle 2 pi U2;
 * disk |v| = 1.5 sqrt(U1), angle 2 pi U2; box v = 1.5 (2 U1 - 1, 2 U2 - 1).
 *   u_dev:     device, 2n floats in [0, 1] (U1, U2 per sample)
 *   m_out_dev: device, 2n floats (s, t per sample)
 *   tri_out_dev (nullable): device, n triangle ids 2 (j (N-1) + i) + (0 | 1), or ~0u
 *   flags_out_dev (nullable): device, n PNDF_SF_* words
 * Asynchronous on stream.  Errors: INVALID_ARG (null or misaligned pointers,
 * n < 0, kernel, jac_eps outside 0 or [1e-9, 1e-2]), CUDA.
 */
pndf_status pndf_sample_normals(const pndf_hierarchy *h, const pndf_query *q_dev, const float *u_dev, int64_t n,
                                int32_t kernel, float jac_eps, float *m_out_dev, uint32_t *tri_out_dev,
                                uint32_t *flags_out_dev, void *stream);

/*
 * GGX projected-area fit per mip node (Eq. 12) and the shadow-masking term
 * (Sec. 4.3).  P'(w) = (w_z + sqrt(w_z^2 + w_xy^T Omega w_xy)) / 2 (Eq. 12
 * with its parentheses restored: the GGX projected area), so Lambda'(w) =
 * P'(w) / w_z - 1 is the GGX Smith Lambda of Omega.  Each node of levels 2..L
 * whose quads all lie in the map is box-filtered over its own quads (for
 * which Eq. 9-11 are exact); its projected area at 16 directions (azimuths
 * 2 pi k / 16 at w_z = 0.3) gives (2 P - w_z)^2 - w_z^2 = w_xy^T Omega w_xy,
 * fitted by least squares.  A footprint (x, S) takes the two mip levels
 * around log2(sqrt(12) max(sqrt(S_xx), sqrt(S_yy))) (clamped to [2, L]),
 * each bilinear between node centres (nodes without a fit drop out).
 */
typedef struct pndf_ggx pndf_ggx;

/* Fit every node of h (reads its texels during the call's work on stream).
 * 16 bytes per node of levels >= 2; temporary scratch 128 bytes per leaf
 * block.  Errors: INVALID_ARG, OOM, CUDA. */
pndf_status pndf_ggx_create(const pndf_hierarchy *h, void *stream, pndf_ggx **out);
void pndf_ggx_free(pndf_ggx *g);

/* Lambda'(omega) per record of q_dev (x and S used) and unit direction
 * omega_dev (3 floats, w_z > 0); NaN where no fit covers the footprint.
 * Asynchronous on stream.  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_ggx_lambda(const pndf_ggx *g, const pndf_query *q_dev, const float *omega_dev, int64_t n,
                            float *lambda_out_dev, void *stream);

/* Height-correlated shadow-masking G = H(m~.wi) H(m~.wo) / (1 + Lambda'(wi)
 * + Lambda'(wo)) per record (m = (ms, mt) lifted to the hemisphere), wi/wo
 * 3 floats each (z > 0).  Asynchronous.  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_shadow_masking(const pndf_ggx *g, const pndf_query *q_dev, const float *wi_dev,
                                const float *wo_dev, int64_t n, float *G_out_dev, void *stream);

/* Level l (2..L) of the fit, row-major (J, I), 3 floats per node
 * (O_xx, O_xy, O_yy; NaN without a fit).  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_ggx_level(const pndf_ggx *g, int32_t level, float *omega_out_dev, void *stream);

/* Copy out level l (2 <= l <= L, 2^L >= N-1) of the cluster hierarchy
 * (Sec. 4.2, Eq. 7-8) for inspection, nodes in row-major order (J, I),
 * S = 2^(L-l) per side:
 *   records_dev: device, S*S*8 floats per node (c00.s, c00.t, d10.s, d10.t,
 *                d01.s, d01.t, d11.s, d11.t), corner normals c = c00 + d;
 *   residual_dev: device, S*S floats, e (+inf: no cluster, the node has a
 *                quad outside the map).
 * Asynchronous on stream.  Errors: INVALID_ARG (level, null or misaligned
 * pointers), UNSUPPORTED (built without clusters), CUDA. */
pndf_status pndf_cluster_level(const pndf_hierarchy *h, int32_t level, float *records_dev, float *residual_dev,
                               void *stream);

/*
 * Batched P-NDF evaluation, Eq. 5 (the exact solution of Eq. 2):
 *   D(m, x) = sum over triangles abc with m in n(abc) of
 *             k_r(a l0 + b l1 + c l2 - x) / |(n_b - n_a) x (n_c - n_a)|,
 *   (l0, l1, l2) = bary(m, n(abc)) (Tab. 1).
 * The hit test is closed (all barycentrics >= 0, m inside the closed normal
 * bounding box); zero-area normal triangles are skipped (a delta, not a
 * density); triangles of normal-space area below 1e-10 are tested and
 * weighted in FP64, all others in FP32.  The pyramid only prunes, so the set
 * of contributing triangles equals that of the flat mode.  Each query's sum
 * is exact: every contribution is rounded once to a multiple of 2^-64 and
 * added in 128-bit fixed point, and the total is rounded to FP32 once, so D
 * does not depend on the order of the hits, on the batch, the launch shape or
 * the division of a large footprint among warps (D = +inf if a sum reaches
 * 2^63, only possible for normal triangles of area far below 1e-20).
 *   q_dev:          device, nq pndf_query records.
 *   D_out_dev:      device, nq floats, caller order.
 *   flags_out_dev:  device, nq uint32 (PNDF_QF_* bits) or NULL.
 *   stats_dev:      device, nq pndf_query_stats or NULL.
 * nq = 0 is valid and launches nothing.  Scratch memory for the key sort
 * (8 bytes per query plus a histogram of 16 KiB to 1 MiB) and for dividing
 * large footprints (1 byte per query plus about 1.7 MB) is allocated
 * stream-ordered from the device's default memory pool and released on the
 * same stream.
 * Errors: INVALID_ARG, OOM, CUDA.  Invalid queries give D = NaN and set
 * PNDF_QF_INVALID (and the device status word).
 */
pndf_status pndf_eval_batch(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq,
                            float *D_out_dev, uint32_t *flags_out_dev, pndf_query_stats *stats_dev,
                            void *stream);

/* pndf_eval_batch with explicit mode, sorting and launch shape (cfg may be
 * NULL for the defaults). */
pndf_status pndf_eval_batch_ex(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq,
                               float *D_out_dev, uint32_t *flags_out_dev, pndf_query_stats *stats_dev,
                               const pndf_eval_config *cfg, void *stream);

/*
 * Allocation-free variant of pndf_eval_batch (the paper has no counterpart:
 * this serves callers that may not allocate device memory, such as a
 * renderer plugin whose host owns all device allocations, a real-time thread
 * that cannot take cudaMalloc's device-wide synchronisation, or code with a
 * fixed device-memory budget).  Same result, bit for bit, as
 * pndf_eval_batch with the default configuration (it evaluates every query
 * with one warp, as it has no scratch to divide large footprints), for at
 * most pndf_eval_noalloc_max_queries()
 * (1,048,576) queries per call; larger batches return PNDF_ERR_CAPACITY
 * before any work is queued.  The sort scratch is one fixed device array
 * (about 9.4 MB) that every GPU loading the library holds until the process
 * exits; nothing is allocated or freed.  The first call on each device looks
 * up that array's device address (cudaGetSymbolAddress) with the device
 * current, so make it before any stream capture; after a device reset the
 * first call in the new context looks it up again.  Every call shares the
 * array: calls whose work can overlap on the GPU (another stream, or earlier
 * work still running) race on it and must be serialised by the caller.
 *   flags_out_dev: device, nq uint32 (PNDF_QF_* bits) or NULL.
 * Errors: INVALID_ARG, CAPACITY, CUDA.
 */
pndf_status pndf_eval_batch_noalloc(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq,
                                    float *D_out_dev, uint32_t *flags_out_dev, void *stream);

/* Largest nq that pndf_eval_batch_noalloc accepts. */
int64_t pndf_eval_noalloc_max_queries(void);

/*
 * End-to-end variant with HOST buffers: copies nq queries from q_host to the
 * device, evaluates as pndf_eval_batch, and copies D back to D_host, all on
 * stream; returns after the stream has completed the copy-back.  Pinned host
 * memory gives full copy bandwidth; pageable memory works but is slower.
 * Device staging (36 bytes per query) is allocated stream-ordered.
 */
pndf_status pndf_eval_batch_host(const pndf_hierarchy *h, const pndf_query *q_host, int64_t nq,
                                 float *D_host, void *stream);

/*
 * Analytic projected area P(w) of each footprint (Eq. 9-11, App. B):
 *   P(w) = sum over triangles T of k_r(T) / |(n_b - n_a) x (n_c - n_a)|
 *          * integral over n+(T) of (w_x m~_x / m~_z + w_z) dm
 * in the frame rotated so w_y = 0, with n+(T) the part of the normal
 * triangle whose normals see w (clipped as in Alg. 1) and the integral
 * taken by Stokes over its boundary (Eq. 11, minus sign on the w_x line
 * term).  w is used as the unit vector w / |w|.  k_r(T) is the kernel at T's
 * uv centroid (cut at q > 16).  A triangle whose normals collapsed onto a
 * segment (|cross| < 1e-12) contributes the segment form of Eq. 13: k_r(T)
 * times the uv-triangle integral of max(n~(u).w, 0) / n~_z(u).  Fully
 * visible triangles are integrated in FP32; partly visible ones, long
 * slivers and collapsed ones in FP64.  The aggregated diffuse BRDF is
 * f_d = P / (pi w_z) (Eq. 13) and the shadow-masking Lambda = P / w_z - 1
 * (Sec. 4.3).
 *   q_dev:     device, nq pndf_query (x, y, sxx, sxy, syy used; ms, mt ignored).
 *   omega_dev: device, 3*nq floats, unit directions with w_z > 0.
 *   P_out_dev: device, nq floats.
 * Every triangle of the footprint is integrated (no pruning applies: every
 * visible triangle contributes).  Large footprints are split into tiles whose
 * partial sums are reduced in a fixed order.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
pndf_status pndf_diffuse_projected_area(const pndf_hierarchy *h, const pndf_query *q_dev,
                                        const float *omega_dev, int64_t nq, float *P_out_dev,
                                        void *stream);

/*
 * Evaluation order for a batch (the keying and counting sort that
 * pndf_eval_batch applies internally, App. C entry level): order_dev receives
 * a permutation of 0..nq-1, largest footprints first, grouped by tile.
 *   order_dev: device, nq uint32.  Scratch is stream-ordered from the pool.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
pndf_status pndf_sort_queries(const pndf_hierarchy *h, const pndf_query *q_dev, int64_t nq, uint32_t *order_dev,
                              void *stream);

/* ---------------------------------------------------------------------------
 * Sharding one batch over hierarchy replicas.
 *
 * Queries are independent and a hierarchy is read-only (Sec. 4.2, Eq. 5), so
 * one batch can be split over replicas of the hierarchy (one per device, or
 * several on one device): put the batch in evaluation order once
 * (pndf_sort_queries), cut that order into contiguous ranges of about equal
 * estimated work (pndf_shard_work's per-block sums), gather each range's
 * records into a contiguous array for its replica (pndf_gather_queries),
 * evaluate it there in the given order (pndf_eval_batch_ex with
 * PNDF_SORT_NONE), and scatter the results back into caller order
 * (pndf_scatter_results).  Each query's D is the same whichever shard, batch
 * or launch evaluates it.  These calls move data only; they take device
 * pointers of the current device and run asynchronously on stream.
 * ------------------------------------------------------------------------- */

/* Estimated work of the evaluation order in blocks of `block` positions:
 * partial_out_dev[b] = sum over positions k in [b block, (b + 1) block) of
 * 64 + 64 sigma_x sigma_y for query order_dev[k] (the area of its 4-sigma box
 * in texel^2 plus a fixed descent cost; invalid covariances count 64).
 *   order_dev:       device, nq uint32 (a permutation from pndf_sort_queries)
 *   partial_out_dev: device, ceil(nq / block) doubles
 * Errors: INVALID_ARG (null or misaligned pointers, nq < 0, block outside
 * 256..2^20), CUDA. */
pndf_status pndf_shard_work(const pndf_query *q_dev, const uint32_t *order_dev, int64_t nq, int32_t block,
                            double *partial_out_dev, void *stream);

/* q_out_dev[k] = q_dev[order_dev[first + k]] for k < count: one range of the
 * evaluation order as a contiguous batch.  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_gather_queries(const pndf_query *q_dev, const uint32_t *order_dev, int64_t first, int64_t count,
                                pndf_query *q_out_dev, void *stream);

/* D_out_dev[order_dev[first + k]] = D_shard_dev[k] for k < count: a range's
 * results put back in caller order.  Errors: INVALID_ARG, CUDA. */
pndf_status pndf_scatter_results(const float *D_shard_dev, const uint32_t *order_dev, int64_t first, int64_t count,
                                 float *D_out_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching over several resident hierarchies.
 *
 * A server holds a table of hierarchies (same texel and bounds formats) and
 * runs steps.  A step evaluates a list of segments, each a slice of one
 * request's queries on one map, in a single persistent kernel launch: warps
 * pull queries from all segments through one work cursor, so requests of
 * different sizes and maps share the GPU.  Each step is a CUDA graph (copy of
 * the segment table from pinned host memory, cursor reset, kernel) replayed
 * with new table contents; table slots rotate, so the host can queue
 * several steps while earlier ones run.  Footprints far larger than the
 * step's average share per warp are divided among warps as in
 * pndf_eval_batch.  A query's result does not depend on which other segments
 * share its step (its sum is exact): it equals pndf_eval_batch's bit for bit.
 * ------------------------------------------------------------------------- */

typedef enum pndf_segment_kind {
    PNDF_SEGMENT_PNDF = 0,            /* P-NDF queries (Eq. 5)                                */
    PNDF_SEGMENT_PROJECTED_AREA = 1   /* projected-area requests (Eq. 9-11), as               */
                                      /* pndf_diffuse_projected_area evaluates them           */
} pndf_segment_kind;

typedef struct pndf_segment {
    const pndf_query *q;    /* device: the request's query records                    */
    const uint32_t *order;  /* device: evaluation order (indices into q), or NULL      */
                            /* (projected area: NULL)                                  */
    float *D;               /* device: the request's results (D, or P), indexed like q */
    uint32_t *flags;        /* device: per-query PNDF_QF_* bits, or NULL (area: NULL)  */
    int32_t map;            /* index into the server's hierarchy table                 */
    int32_t first;          /* first position of this slice (in order[], else in q[])  */
    int32_t count;          /* queries (requests) in this slice                        */
    int32_t kind;           /* pndf_segment_kind                                       */
    const float *omega;     /* projected area: 3 floats per record of q (unit, w_z > 0) */
} pndf_segment;

typedef struct pndf_server pndf_server;

typedef struct pndf_server_config {
    int32_t max_segments;   /* segments per step (0 = 1024)                           */
    int32_t warps_per_cta;  /* 0 = 8                                                  */
    int32_t ctas_per_sm;    /* 0 = as many as fit                                     */
    int32_t slots;          /* table slots, 2..8 (0 = 4): steps that can be queued     */
    int32_t kernel;         /* footprint kernel (pndf_kernel) of every query served   */
    float tau;              /* > 0: the cluster cut of Sec. 4.2 (Gaussian kernel only;
                               every map built with clusters = 1)                     */
    float jac_eps;          /* > 0: the Eq. 6 clamp (Gaussian kernel, tau = 0)         */
    int32_t max_area_requests; /* projected-area requests per step, 0..65536 (0: none;
                               their band scratch is reserved per table slot)        */
} pndf_server_config;

/* Create a server over nmaps (1..8) hierarchies on the current device; maps
 * must outlive the server.  Every query it serves is evaluated as
 * pndf_eval_batch_ex evaluates it with the same kernel, tau and jac_eps (the
 * variant is fixed per server: the step graphs capture its kernel).
 * Allocates its tables (device and pinned host) and captures the step graphs.
 * With cfg->max_area_requests > 0 a step can also hold projected-area
 * requests (segment kind PNDF_SEGMENT_PROJECTED_AREA), evaluated in the same
 * step graph by the kernels of pndf_diffuse_projected_area (so P is the same
 * bit for bit as that call gives); each table slot reserves their band
 * scratch, 4 (max + 1) + 8 max B bytes with B = (N_max + 6) / 8 + 1 bands for
 * the largest map side N_max.
 * Errors: INVALID_ARG (formats differ, bad counts, kernel / tau / jac_eps out
 * of range), UNSUPPORTED (tau with a map built without clusters, or with the
 * disk / box kernel or the clamp; the clamp with the disk / box kernel), OOM,
 * CUDA. */
pndf_status pndf_server_create(const pndf_hierarchy *const *maps, int32_t nmaps, const pndf_server_config *cfg,
                               pndf_server **out);

/* Queue one step over nsegs segments (host array, copied before return) on
 * stream; ev_done (optional cudaEvent_t) is recorded when the step's kernel
 * completes.  Blocks only if the next table slot is still in use by the step
 * queued `slots` steps earlier.  All pointers in the segments must stay valid
 * until the step completes.  P-NDF segments are at most max_segments;
 * projected-area segments (no order or flags, omega required) hold at most
 * max_area_requests requests in total.  Errors: INVALID_ARG (bad map index,
 * kind, count, pointers, too many P-NDF segments), CAPACITY (too many
 * projected-area requests), UNSUPPORTED (projected-area segments on a server
 * created without max_area_requests), CUDA. */
pndf_status pndf_server_step(pndf_server *srv, const pndf_segment *segs_host, int32_t nsegs, void *stream,
                             void *ev_done);

/* Wait for every queued step of this server. */
pndf_status pndf_server_sync(pndf_server *srv);

/* Release the server (waits for its queued steps; safe on NULL). */
void pndf_server_destroy(pndf_server *srv);

/* Read and clear the per-device status word that kernels set on device-side
 * errors, whichever hierarchy and stream they ran on (synchronises stream).
 * PNDF_OK if none; PNDF_ERR_DEVICE otherwise, with the raw PNDF_QF_* bits in
 * *bits_out when bits_out != NULL.  The read and the clear are one atomic
 * exchange on the device, so bits set by kernels still running on other
 * streams are kept for the next read.  Every caller on the device shares
 * this word; pndf_last_device_status reads one hierarchy's own. */
pndf_status pndf_device_status(void *stream, uint32_t *bits_out);

/* Read and clear hierarchy h's own status word (Sec. 4.2's evaluation has no
 * error channel of its own; this is the library's): the PNDF_QF_* bits that
 * kernels recorded while evaluating P-NDF queries or projected areas on h
 * (invalid covariance, traversal stack overflow), on any stream.  Waits for
 * the work queued on stream, then takes the word with one atomic exchange on
 * the device.  Call with h's device current.  PNDF_OK if no bit is set;
 * PNDF_ERR_DEVICE otherwise, with the bits in *bits_out (nullable).
 * Errors: INVALID_ARG (null h, wrong device current), CUDA. */
pndf_status pndf_last_device_status(const pndf_hierarchy *h, void *stream, uint32_t *bits_out);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads); lets a caller count the kernels of a region. */
int64_t pndf_launch_count(void);

/* Static, human-readable name of a status code. */
const char *pndf_status_string(pndf_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t pndf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PNDF_H */
