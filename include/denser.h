/*
 * denser.h -- C ABI of the DENSER hot path on one GPU (sm_103a).
 *
 * The library fuses depth maps into a truncated signed-distance field held in
 * a hashing voxel grid of 8x8x8 voxel blocks, and regularises it with the
 * Omega-aware total-variation primal-dual solver of the paper
 * (Tanner, Pinies, Paz, Newman: "DENSER Cities", Section III).
 *
 * Conventions
 *   - Camera frame: x right, y down, z forward.  A pose T_gc is a 4x4 float64
 *     row-major matrix mapping camera coordinates to global coordinates.
 *   - Voxel (i, j, k) has its centre at ((i+0.5)s, (j+0.5)s, (k+0.5)s), s the voxel
 *     size.  It lives in block (floor(i/8), floor(j/8), floor(k/8)) at local offset
 *     l = lx + 8*ly + 64*lz, lx = i - 8*floor(i/8).
 *   - A block is identified by (segment, bx, by, bz); blocks of different segments
 *     are never neighbours.  segment in [0, 126]; |bx|, |by|, |bz| < 2^18.
 *   - Per-voxel fields are stored block-major: field[block][512].  The dual field p
 *     is stored component-major: p[3][block][512].
 *   - Block indices: every allocation call appends its new blocks in ascending
 *     (segment, bz, by, bx) order, after all blocks allocated earlier (a batched call,
 *     denser_integrate_batch, orders them by the first depth map that reached them,
 *     then by key: the order one call per map gives).
 *   - Depth maps are float32 [height][width]; a pixel is valid when finite and > 0.
 *
 * Pointers
 *   Every buffer argument may be device memory or host memory (pinned or
 *   pageable); the library looks the pointer up with cudaPointerGetAttributes and
 *   stages host memory through its own device buffers.  The caller owns every
 *   buffer it passes; the context owns the hash table, the block pool and the
 *   primal-dual state.  Host depth maps are copied on a stream of the context's own
 *   (into one of two buffers, so that a frame's copy overlaps the previous frame's
 *   kernels) and the call's stream waits for that copy: like any asynchronous copy
 *   from pinned memory, the host buffer must stay unchanged until the call's stream
 *   has passed the call.
 *
 * Streams and errors
 *   `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls enqueue
 *   work on it and return without waiting unless stated.  Every call returns 0
 *   (DENSER_OK) or a negative DENSER_ERR_* code and sets a message readable with
 *   denser_last_error.  Argument errors leave the context unchanged.  Errors
 *   detected on the device (hash or pool full, coordinates out of range, a wait
 *   that ran out) are sticky: they are reported by the next call that waits for
 *   the stream (denser_sync, denser_alloc_blocks with n_new_out, denser_regularize,
 *   denser_energy, denser_extract*, denser_load_*) and are cleared by denser_reset.
 *   A context is used by one host thread at a time.
 */
#ifndef DENSER_H
#define DENSER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DENSER_OK 0
#define DENSER_ERR_INVALID_ARG (-1)
#define DENSER_ERR_HASH_FULL (-2)   /* a key found no free slot within the probe limit */
#define DENSER_ERR_POOL_FULL (-3)   /* more blocks than max_blocks (or max_new_blocks per call) */
#define DENSER_ERR_CUDA (-4)        /* a CUDA runtime call failed; see denser_last_error */
#define DENSER_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define DENSER_ERR_RANGE (-6)       /* a block coordinate outside +-2^18 or a bad segment */
#define DENSER_ERR_TOO_LARGE (-7)   /* more blocks than denser_energy_noalloc can hold */

#define DENSER_FP32 0
#define DENSER_FP16 1
#define DENSER_BF16 2

typedef struct denser_ctx denser_ctx;

/* Method constants and capacities.  Defaults (denser_default_params): Table I of
 * the paper, 10 cm voxels: lambda 0.8, sigma 0.5, tau 1/6, theta 1.0; mu 0.3 m. */
typedef struct {
    double voxel_size;        /* s, metres */
    double mu;                /* truncation distance behind the surface, metres (Eq. 1) */
    double lambda;            /* data-term weight (Eq. 2) */
    double sigma;             /* dual step sigma_p (Section III-C, step 2) */
    double tau;               /* primal step (Section III-C, step 3) */
    double theta;             /* relaxation (Section III-C, step 4) */
    uint32_t hash_slots;      /* power of two, > max_blocks */
    uint32_t max_blocks;      /* block pool capacity, at most 2^24 (voxel offsets are 64-bit) */
    uint32_t max_new_blocks;  /* new blocks one allocation call may add (0: max_blocks) */
    int32_t precision;        /* DENSER_FP32 / FP16 / BF16 storage of u, u_bar, p */
    int32_t gap_every;        /* evaluate the primal-dual gap every this many iterations (0: never) */
    int32_t reserved;
} denser_params;

typedef struct {
    double fx, fy, cx, cy;    /* pixels; pixel (x, y) covers [x, x+1) x [y, y+1) */
    int32_t width, height;    /* each at most 2^20, width * height < 2^31 */
} denser_intrinsics;

typedef struct {
    int32_t iters;            /* iterations run by this call */
    int32_t converged;        /* 1 when gap/|primal| <= gap_tol was reached */
    double primal;            /* P(u) after the last iteration (FP64 reduction) */
    double dual;              /* D(p) after the last iteration */
    double gap;               /* primal - dual */
    double rel_gap;           /* gap / |primal| */
    double sweep_ms;          /* device time of the iteration loop (CUDA events): the sweeps, plus the
                                 gap evaluations when they run inside the graph-captured loop */
    double total_ms;          /* device time of the whole call */
    int32_t sweep_launches;   /* sweep kernel launches timed in sweep_ms */
    int32_t gap_evals;        /* gap evaluations done inside the loop */
    int64_t n_blocks;         /* allocated blocks */
    int64_t n_omega;          /* voxels in Omega (observed) */
} denser_reg_stats;

/* Launch schedule of the primal-dual sweep.  Every schedule computes the same
 * iterates; only speed differs (chosen by the autotuner).
 *   sweep_kernel  0: staged (each CTA loads a block, then computes it),
 *                 1: pipelined (cp.async prefetch of the next block while computing),
 *                 2: rows (one thread per 8-voxel x-row, vector loads),
 *                 3: rows with the next block's own fields prefetched by 1-D bulk copies
 *                    (TMA) into a double-buffered shared-memory stage,
 *                 4: rows with the halos (faces, edges, x halos) copied asynchronously
 *                    (cp.async) into shared memory while the block's own rows load,
 *                 5: as 4, and each thread's row of the next block's own fields is
 *                    copied (cp.async) into a shared-memory slot of its own while the
 *                    current block computes,
 *                 6: software-pipelined rows: the next block's halos (cp.async, into a
 *                    second tile set) and own rows (into registers) are in flight while
 *                    the current block computes,
 *                 7: as 4 with the face and edge halos split into balanced items over
 *                    all 64 threads (82 row items: two per thread for 18 threads, one
 *                    for the rest) instead of one branch per face; the default, with
 *                    order 0 and ctas_per_sm 2,
 *                 8: as 2 with the same balanced face items,
 *                 9: as 6 with the balanced face items
 *   order         0: blocks in index order, 1: blocks sorted by (segment, bz, by, bx)
 *                 (neighbours are visited close together, so halos hit in L2)
 *   ctas_per_sm   resident CTAs per SM for the persistent grid (0: kernel default); for
 *                 the row kernels (2, 4, 7, 8) it picks the register budget: 0/1 -> 8 CTAs of
 *                 64 threads per SM, 2 -> 10, 3 -> 12 (kernel 5: 2 -> 10, else 8; kernels 6
 *                 and 9: 1 -> 5, 3 -> 7, else 6); for kernel 3 it caps CTAs at 2x this
 *   use_graph     1: the iteration loop of denser_regularize runs as one CUDA graph: a
 *                 WHILE conditional node whose body is gap_every sweeps (10 when no gap
 *                 test is asked for) plus the FP64 gap evaluation, and whose condition is
 *                 set on the device (no host round trip per gap test).  The graph is
 *                 recorded once and reused while the map, schedule and loop shape stay
 *                 the same.  Needs an even gap_every; otherwise, and for the iterations
 *                 left over after the last full body pass, sweeps are launched one by one.
 *                 0: one launch per sweep and a host round trip per gap test. */
typedef struct {
    int32_t sweep_kernel;
    int32_t order;
    int32_t ctas_per_sm;
    int32_t use_graph;
} denser_schedule;

/* Fills *p with the defaults above (hash 2^20 slots, 65536 blocks, FP32). */
void denser_default_params(denser_params* p);

/* Creates a context on CUDA device `device` and allocates its pool, hash table and
 * state (about 46 B x 512 per block of capacity in FP32).  *out receives the context. */
int denser_create(const denser_params* params, int32_t device, denser_ctx** out);

/* Frees the context and everything it owns.  NULL is ignored. */
void denser_destroy(denser_ctx* ctx);

/* Empties the map (no blocks), zeroes the state and clears sticky errors. */
int denser_reset(denser_ctx* ctx, void* stream);

/* Message of the last error on this context ("" if none).  Valid until the next call. */
const char* denser_last_error(const denser_ctx* ctx);

/* Waits for `stream` and returns the sticky device error, if any. */
int denser_sync(denser_ctx* ctx, void* stream);

/* Allocation (Section III-A, "Fusing Data"): every block that holds a sample of a
 * valid pixel's ray at depths z = d + n*s/2, n = -N..N, N = ceil(mu/(s/2)), z > 0,
 * is allocated (f = w = 0) if absent.  Each block key is the floor of a float64
 * expression written out in a fixed operation order; the kernel evaluates it in float32
 * with a forward error bound and recomputes it in float64, in that order, wherever the
 * bound cannot certify the floor, so block sets and indices are exact.
 * depth: float32 [height][width]; K: intrinsics; T_gc: 16 float64 (host memory);
 * segment: block-key segment.  n_new_out (host, may be NULL): number of new blocks;
 * when non-NULL the call waits for the stream. */
int denser_alloc_blocks(denser_ctx* ctx, const float* depth, const denser_intrinsics* K,
                        const double T_gc[16], int32_t segment, void* stream,
                        int32_t* n_new_out);

/* Projective fusion, Eq. 1 (Section III-A, steps 1-4): every allocated voxel of
 * `segment` is projected into the depth map (nearest pixel = floor of the
 * projection); where the pixel is valid and u_SDF = d - z_c >= -mu, w += 1 and
 * f = (min(1, u_SDF/mu) + w_old f_old) / w.  The update decision (pixel index and
 * the u_SDF >= -mu test) is that of the float64 expressions in a fixed operation
 * order: the kernel takes it in float32 with a per-voxel error bound and recomputes it
 * in float64 wherever the bound cannot certify it, so w is exact; f is accumulated in
 * float32. */
int denser_fuse_depth(denser_ctx* ctx, const float* depth, const denser_intrinsics* K,
                      const double T_gc[16], int32_t segment, void* stream);

/* denser_alloc_blocks followed by denser_fuse_depth on the same depth map, which is
 * staged once when it is in host memory.  Arguments and results as those two calls. */
int denser_integrate(denser_ctx* ctx, const float* depth, const denser_intrinsics* K,
                     const double T_gc[16], int32_t segment, void* stream, int32_t* n_new_out);

/* Allocation and fusion (Section III-A, Eq. 1) of n_frames depth maps of one camera, in
 * order: the same result as n_frames calls of denser_integrate (the same blocks, block
 * indices, f and w, bit for bit), in one allocation pass and one fusion pass per
 * DENSER_MAX_BATCH maps.  A block first
 * reached by map i is indexed after every block first reached by an earlier map, as
 * one call per map gives, and takes maps i, i+1, ... only; each voxel takes its maps
 * in order, so the running mean of Eq. 1 sees the same operands.
 * depths: float32 [n_frames][height][width], host or device memory (host maps are
 * staged DENSER_MAX_BATCH at a time); T_gc: float64 [n_frames][16] in host memory.
 * n_new_out (host, may be NULL): blocks added by the whole call; when non-NULL the
 * call waits for the stream after each group of maps.  An error stops the call after
 * the group it occurred in; the sticky device error is reported by denser_sync. */
#define DENSER_MAX_BATCH 16
int denser_integrate_batch(denser_ctx* ctx, const float* depths, int32_t n_frames, const denser_intrinsics* K,
                           const double* T_gc, int32_t segment, void* stream, int32_t* n_new_out);

/* ------------------------------------------------------------------ laser scans
 * The projective update extends to laser sensors by updating only the voxels along
 * each ray, from the sensor to mu behind the observed surface (Section III-A, after
 * Eq. 1).  points: float32 [n_points][3] in the sensor frame (host or device memory);
 * T_gs: 16 float64 (host), sensor -> global, rotation R and origin t.  A point is valid
 * when finite, at range r = |p| > 0 and with floor((r + mu) / (s/2)) < 2^22; others are
 * skipped.  Ray direction dg = R p / r, every float64 step in the oracle's order.
 *
 * denser_alloc_points: blocks holding a band sample at range r + n s/2, n = -N..N,
 *   N = ceil(mu / (s/2)), range > 0, are allocated (the rule of denser_alloc_blocks along
 *   the ray); new blocks are appended in ascending (segment, bz, by, bx) order.
 * denser_fuse_points: every voxel of an allocated block of `segment` holding a ray sample
 *   at range n s/2, n = 0..floor((r + mu)/(s/2)), counts once per ray; it observes
 *   u_SDF = r - (c - t) . dg (c its centre) when u_SDF >= -mu.  The scan updates each
 *   voxel once: w += n_obs, f = (w_old f_old + sum min(1, u_SDF/mu)) / w, the sum in
 *   fixed point (multiples of 2^-30), so that the result does not depend on ray order.
 *   Block sets and w are bit-exact with the oracle; f carries float32 rounding.
 * denser_integrate_points: both, with one staging of host points.
 * n_new_out (host, may be NULL): new blocks; when non-NULL the call waits. */
int denser_alloc_points(denser_ctx* ctx, const float* points, int64_t n_points, const double T_gs[16],
                        int32_t segment, void* stream, int32_t* n_new_out);
int denser_fuse_points(denser_ctx* ctx, const float* points, int64_t n_points, const double T_gs[16],
                       int32_t segment, void* stream);
int denser_integrate_points(denser_ctx* ctx, const float* points, int64_t n_points, const double T_gs[16],
                            int32_t segment, void* stream, int32_t* n_new_out);

/* ------------------------------------------------------------------ stereo depth maps
 * Depth-map estimation from a rectified pair (Section IV): a Census Transform Signature
 * data term (IV-A) and an affine TGV regulariser shaped by an image-driven diffusion
 * tensor (IV-B, IV-C).  The paper fixes no window, range or optimiser schedule; here:
 * I_R is the reference (rho compares I_L(x + d, y) with I_R(x, y)), a 9 x 7 Census
 * window (62 bits, edge pixels repeated), cost = Hamming / 62 (1 off the image),
 * T = I + (exp(-gamma |grad I_R|^beta) - 1) n n^T, and the data term decoupled by an
 * auxiliary field a: `outer` times an exhaustive integer a-step (argmin over delta in
 * [0, max_disp) of lambda C + (d - delta)^2 / (2 theta), float32, ties to the smaller
 * delta) then `inner` Chambolle-Pock iterations on the TGV-L2 problem, theta shrinking
 * by theta_decay.  Images are float32 [height][width] in [0, 1]; every pointer of these
 * calls is device memory (host pointers are DENSER_ERR_INVALID_ARG); width, height >= 2.
 * They need no context, enqueue on `stream` and do not wait. */
typedef struct {
    int32_t max_disp;                 /* disparities 0 .. max_disp - 1 */
    float lambda, alpha1, alpha2;     /* Table I: 0.5, 1.0, 5.0 */
    float beta, gamma;                /* Table I: 1.0, 4.0 */
    float theta0, theta_decay;        /* coupling schedule: 2.0, 0.5 */
    int32_t outer, inner;             /* 8 a-steps, 80 primal-dual iterations after each */
} denser_stereo_params;

void denser_stereo_default_params(denser_stereo_params* p);

/* 62-bit Census signatures sig uint64 [h][w] of img (bit b: the b-th window pixel in
 * row-major order, the centre skipped, is darker than the centre). */
int denser_census(const float* img, int32_t width, int32_t height, uint64_t* sig, void* stream);

/* Diffusion tensor of img as three planes float32 [3][h][w]: t00, t01 (= t10), t11. */
int denser_diffusion_tensor(const float* img, int32_t width, int32_t height, float gamma, float beta,
                            float* tensor, void* stream);

/* a-step: a = argmin_delta lambda Hamming/62 + (d - delta)^2 / (2 theta) per pixel
 * (a float32 [h][w] holds integers); theta <= 0 or infinite drops the coupling; a may
 * alias d. */
int denser_disparity_assign(const uint64_t* sig_left, const uint64_t* sig_right, int32_t width,
                            int32_t height, int32_t max_disp, float lambda, double theta,
                            const float* d, float* a, void* stream);

/* `iters` primal-dual iterations of the d-step on state float32 [24][h][w]: the first 12
 * planes hold d, d_bar, w1, w2, w_bar1, w_bar2, p1, p2, q11, q12, q21, q22 (in that
 * order) on entry and on return; the last 12 are working space. */
int denser_tgv_iterate(const float* a, const float* tensor, int32_t width, int32_t height, float alpha1,
                       float alpha2, double theta, int32_t iters, float* state, void* stream);

/* Bytes of workspace denser_stereo_estimate needs for a width x height pair. */
size_t denser_stereo_workspace_size(int32_t width, int32_t height);

/* The whole estimate: disparity float32 [h][w] on I_R's grid. */
int denser_stereo_estimate(const float* img_left, const float* img_right, int32_t width, int32_t height,
                           const denser_stereo_params* params, void* workspace, size_t workspace_bytes,
                           float* disparity, void* stream);

/* depth = fx * baseline / disparity where disparity > min_disp, else 0 (invalid), the
 * depth-map input of denser_alloc_blocks / denser_fuse_depth / denser_integrate. */
int denser_disparity_to_depth(const float* disparity, int32_t width, int32_t height, float fx, float baseline,
                              float min_disp, float* depth, void* stream);

/* Regularisation (Section III-B/C): Chambolle-Pock iterations on the Omega-aware
 * TV-L2 energy over the allocated blocks, Omega = {w > 0}:
 *   p <- P(p + sigma grad_Omega u_bar),  P(q) = q / max(1, |q|_2)   (grad_Omega: Eq. 3)
 *   u <- (u + tau div_Omega p + tau lambda w f) / (1 + tau lambda w) on Omega (div_Omega: Eq. 4)
 *   u_bar <- u + theta (u - u_old)
 * start: 0 = from p = u = u_bar = 0 (step 1), 1 = resume from the current state.
 * Runs max_iters iterations, or stops earlier once gap/|P| <= gap_tol (gap_tol > 0
 * and params.gap_every > 0).  Waits for the stream when `out` is non-NULL or a gap
 * check is due; `out` (host, may be NULL) receives the statistics. */
int denser_regularize(denser_ctx* ctx, int32_t max_iters, double gap_tol, int32_t start,
                      void* stream, denser_reg_stats* out);

/* FP64 primal and dual energies of the current state (waits for the stream):
 *   P(u) = sum_Omega |grad u|_2 + (lambda/2) sum_Omega w (u - f)^2
 *   D(p) = sum_Omega [ -f div p - (div p)^2 / (2 lambda w) ]
 * (Section III-B, Eq. 2 with the weighting of the update, and its dual).  Sums and
 * terms in float64; each |grad u|_2 is a float32 reciprocal square root refined by one
 * float64 Heron step (relative error below 2^-40), and 1/(2 lambda w) for integer counts
 * w <= 4096 comes from a table of float64 quotients.  primal, dual: host pointers
 * (either may be NULL). */
int denser_energy(denser_ctx* ctx, double* primal, double* dual, void* stream);

/* Copies the map out in block-index order (waits for the stream).  Any output may
 * be NULL.  coords: int32 [n][4] (segment, bx, by, bz); f, w, u: float32 [n][512];
 * omega: uint8 [n][512] (1 = observed).  capacity_blocks: rows the outputs hold;
 * fewer than the map's blocks is DENSER_ERR_INVALID_ARG.  n_blocks_out: host. */
int denser_extract(denser_ctx* ctx, int32_t* coords, float* f, float* w, uint8_t* omega,
                   float* u, int64_t capacity_blocks, int64_t* n_blocks_out, void* stream);

/* Copies the relaxed primal u_bar [n][512] and the dual p [3][n][512] out (float32,
 * converted from the storage precision).  Either may be NULL. */
int denser_extract_dual(denser_ctx* ctx, float* u_bar, float* p, int64_t capacity_blocks,
                        void* stream);

/* Surface extraction: the zero level set of u over the observed voxels, as a list of
 * triangles.  The paper's pipeline extracts a surface from the regularised model for
 * other components (Section II, Fig. 1) but names no method; this one meshes each cube
 * of 2x2x2 voxel centres whose eight corners are observed (w > 0), split into the six
 * Kuhn tetrahedra around its main diagonal, with a vertex at the linear zero of u on
 * every tetrahedron edge whose ends differ in sign (u < 0 negative, u >= 0 not).
 * Triangles are wound so that (v1 - v0) x (v2 - v0) points to the side u >= 0, and are
 * ordered by block index, cube (lower corner's local index), tetrahedron, triangle.
 *   tri_pos  float32 [capacity][3][3]: vertex world positions in metres (voxel (i,j,k)
 *            has its centre at ((i,j,k) + 1/2) voxel_size in its segment's frame);
 *   tri_ids  int64 [capacity][3]: vertex ids, (flat voxel index of the edge's lower end
 *            = block * 512 + local index) * 8 + direction bits (1 +x, 2 +y, 4 +z); equal
 *            ids are the same vertex.
 *   block_first  int64 [n_blocks + 1]: index of each block's first triangle (the
 *            triangles of block b, those whose cube has its lower corner in b, are
 *            [block_first[b], block_first[b + 1])), block_first[n_blocks] = total.
 * Any of the three may be NULL (all NULL counts only); each may be host or device
 * memory (host triangle buffers are staged through device scratch the context keeps).
 * *n_tri_out (host, required) receives the total number of triangles.  The call waits
 * for the stream.  When the total exceeds capacity, the first `capacity` triangles are
 * written and DENSER_ERR_TOO_LARGE is returned (block_first is complete either way). */
int denser_extract_surface(denser_ctx* ctx, float* tri_pos, int64_t* tri_ids, int64_t capacity,
                           int64_t* n_tri_out, int64_t* block_first, void* stream);

/* Appends n blocks with the given coordinates (int32 [n][4]) and fusion state
 * (f, w float32 [n][512]; NULL = zeros) in the given order, with zero primal-dual
 * state.  A coordinate already in the map is DENSER_ERR_INVALID_ARG. */
int denser_load_blocks(denser_ctx* ctx, const int32_t* coords, const float* f, const float* w,
                       int64_t n, void* stream);

/* Overwrites the primal-dual state of all n = n_blocks blocks: u, u_bar [n][512],
 * p [3][n][512] float32 (converted to the storage precision).  NULL = zeros. */
int denser_load_state(denser_ctx* ctx, const float* u, const float* u_bar, const float* p,
                      int64_t n, void* stream);

/* Sets / reads the sweep schedule (see denser_schedule).  Out-of-range fields are
 * DENSER_ERR_INVALID_ARG. */
int denser_set_schedule(denser_ctx* ctx, const denser_schedule* sch);
int denser_get_schedule(const denser_ctx* ctx, denser_schedule* sch);

/* Fusion profile: device times of the allocation and fusion kernels of
 * denser_integrate_batch, measured with CUDA events while profiling is on.  With
 * profiling on, every batched call waits for its stream after each group of maps (to
 * read the events and counters), so the profile is for measurement, not for the
 * fastest pipeline.  Totals since profiling was last switched on: */
typedef struct {
    int64_t groups;           /* groups of up to DENSER_MAX_BATCH maps (one launch sequence each) */
    int64_t maps;             /* depth maps */
    int64_t listed_blocks;    /* sum over groups of the blocks the culling listed for the fusion kernel */
    int64_t new_blocks;       /* blocks the allocation added */
    double key_pass_ms;       /* the key pass: one thread per pixel, band samples, hash inserts */
    double alloc_rest_ms;     /* sort, index, zero and commit of the new keys */
    double cull_ms;           /* culling and per-map block origins */
    double fuse_ms;           /* the fusion kernel: Eq. 1 on every listed voxel, maps in order */
} denser_fusion_profile;

/* Switches fusion profiling on (1; the totals restart at zero) or off (0). */
int denser_set_fusion_profiling(denser_ctx* ctx, int32_t enable);
/* Copies the totals accumulated since profiling was switched on. */
int denser_get_fusion_profile(const denser_ctx* ctx, denser_fusion_profile* out);

/* Number of allocated blocks (waits for the stream); negative on error. */
int64_t denser_num_blocks(denser_ctx* ctx, void* stream);

/* Kernels this context has launched since it was created. */
uint64_t denser_launch_count(const denser_ctx* ctx);

/* ------------------------------------------------------------------ warm start
 * A small 3D convolutional network gives the primal-dual iteration a starting point
 * (the paper starts from zero, Section III-C step 1; the network is not part of it).
 * Inputs are a block and its one-voxel halo, 10^3 voxels; outputs the block's 8^3
 * (u, p_x, p_y, p_z).  Four 3^3 convolutions with zero padding over the 10^3 grid,
 * ReLU after the first three.  Tensors, all in device memory:
 *   activations  BF16 [n][1000][16], voxel x + 10 y + 100 z of the 10^3 grid, channel last
 *                (the input uses channels 0 = f, 1 = w / (w + 8); the output channels 0..3)
 *   weights      BF16 [27][16 out][16 in], tap dx + 3 dy + 9 dz for offset (dx-1, dy-1, dz-1)
 *   biases       FP32 [16]
 * Products run on tensor cores (BF16 inputs, FP32 accumulation).  `blocks` lists block
 * indices (device int32 [n]); NULL means blocks 0..n-1. */

/* Network inputs of the listed blocks: x BF16 [n][1000][16]. */
int denser_net_gather(denser_ctx* ctx, const int32_t* blocks, int64_t n, void* x, void* stream);

/* Training targets from the context's current state: target FP32 [n][4][512] (u, p_x,
 * p_y, p_z) and mask FP32 [n][4][512]: sqrt(u_weight) where the voxel is in Omega (u),
 * sqrt(p_weight) where the Eq. 3 edge along axis a exists (p_a), 0 elsewhere, so that the
 * loss of denser_net_loss weighs squared errors of u and p by u_weight and p_weight. */
int denser_net_targets(denser_ctx* ctx, const int32_t* blocks, int64_t n, float* target, float* mask,
                       float u_weight, float p_weight, void* stream);

/* Divergence targets from the context's current state: target FP32 [n][6][512], channels
 * 0 u (0 off Omega), 1 Omega (1 or 0), 2 the divergence of p over the block's inner Eq. 3
 * edges (Eq. 4 with the edges that cross the block's faces left out; 0 off Omega), 3..5
 * the inner edge masks e_a = Omega(l) and Omega(l + a) and l_a < 7, for the loss of
 * denser_net_loss_div.  The dual field is unique only up to a divergence-free part;
 * its divergence is what a warm start must get right. */
int denser_net_targets_div(denser_ctx* ctx, const int32_t* blocks, int64_t n, float* target, void* stream);

/* Writes a warm start into the state from network outputs out FP32 [n][1000][16]:
 * u = clamp(out_0, -1, 1) on Omega and 0 elsewhere, u_bar = u, p_a = out_{1+a} on the
 * Eq. 3 edges and 0 elsewhere, then p projected onto the unit ball.  with_dual 0: p = 0
 * everywhere; 1: p on every Eq. 3 edge; 2: p on the edges inside the block only (0 on the
 * edges that cross a block face, the network trained by denser_net_loss_div).  Follow it
 * with denser_regularize(start = 1). */
int denser_net_apply(denser_ctx* ctx, const int32_t* blocks, int64_t n, const float* out, int32_t with_dual,
                     void* stream);

/* One layer: y = conv(x, w) + bias, then ReLU when relu != 0, on the fifth-generation
 * tensor cores (tcgen05.mma, BF16 products accumulated in FP32 in tensor memory; a wait
 * for their completion that runs out is reported by denser_net_check).  x BF16 [n][1000][16];
 * bias FP32 [16] or NULL; outputs y_bf16 BF16 and/or y_f32 FP32 [n][1000][16] (either
 * may be NULL).  The data gradient of a layer is the same call on its output gradient
 * with the mirrored, transposed weights of denser_pack_weights and no bias or ReLU. */
int denser_conv3(const void* x, const void* w, const float* bias, int32_t relu, void* y_bf16, float* y_f32,
                 int64_t n, void* stream);

/* Waits for `stream`; DENSER_ERR_TIMEOUT when a denser_conv3 since the last check gave up
 * waiting for its tensor-core products (its outputs are then incomplete), else DENSER_OK. */
int denser_net_check(void* stream);

/* Weight and bias gradients of a layer, accumulated (+=) into dw FP32 [27][16][16] and
 * db FP32 [16]: dw[tap][co][ci] += sum_n sum_v dz[v][co] h[v + offset(tap)][ci], db[co] +=
 * sum dz[v][co]; h is the layer input and dz the gradient at its pre-activation, BF16. */
int denser_conv3_wgrad(const void* h, const void* dz, float* dw, float* db, int64_t n, void* stream);

/* dz = dh where h > 0, else 0 (BF16, `count` elements): the gradient through a ReLU. */
int denser_relu_backward(const void* dh, const void* h, void* dz, int64_t count, void* stream);

/* Masked squared error of outputs out FP32 [n][1000][16] (channels 0..3 on the centre
 * 8^3) against target/mask FP32 [n][4][512]: *loss += sum mask (out - target)^2 / n
 * (device FP64), dout BF16 [n][1000][16] = its gradient (zero off the centre). */
int denser_net_loss(const float* out, const float* target, const float* mask, void* dout, double* loss,
                    int64_t n, void* stream);

/* Loss of the divergence-trained warm start, for outputs out FP32 [n][1000][16] (u =
 * channel 0, p_a = channel 1 + a on the centre 8^3) and targets FP32 [n][6][512] of
 * denser_net_targets_div:
 *   *loss += (1/n) sum_samples sum_Omega [ u_weight (u - u*)^2 + div_weight (div p - div p*)^2 ]
 * with div the inner-edge divergence (p counted on the inner edges only); dout BF16
 * [n][1000][16] = its gradient (zero off the centre and off channels 0..3).  loss is a
 * device FP64 scalar; every pointer is device memory. */
int denser_net_loss_div(const float* out, const float* target, float u_weight, float div_weight, void* dout,
                        double* loss, int64_t n, void* stream);

/* Adam update of FP32 parameters w with gradient grad and moments m, v (count elements),
 * bias-corrected for step `step` (>= 1). */
int denser_adam(float* w, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                float beta2, float eps, int32_t step, void* stream);

/* BF16 copies of FP32 weights [27][16][16]: wf in the forward layout and wb with taps
 * mirrored and in/out channels swapped (the data-gradient convolution). */
int denser_pack_weights(const float* w32, void* wf, void* wb, void* stream);

/* Energies without allocation.  The paper has no counterpart to this call; it exists
 * for callers that may not allocate device memory: a process whose device memory all
 * belongs to its own allocator (a framework's caching allocator, or the fixed memory
 * budget of an on-vehicle mapping process) must not call cudaMalloc behind it, and a
 * latency-critical loop cannot take the device-wide synchronisation that cudaMalloc
 * and cudaFree may cause.  It computes the same P(u) and D(p) as denser_energy, but
 * from caller-owned buffers and with no context: coords int32 [n][4], f, w, u float32
 * [n][512] and p float32 [3][n][512], all in device memory of the current device (or
 * managed memory), in the layouts that denser_extract and denser_extract_dual write.
 * coords must be 16-byte aligned and the float buffers 4-byte aligned.  out (host
 * memory, or 8-byte aligned device memory of the current device) receives {P, D};
 * with a host `out` the call waits for the stream.
 * Its only working memory is a fixed 2.2 MB array in device memory that every GPU which
 * loads the library holds until the process exits.  That size caps the map at
 * DENSER_NOALLOC_MAX_BLOCKS blocks: a larger n_blocks returns DENSER_ERR_TOO_LARGE.
 * The first call on a device looks the array's address up for that device (a one-time
 * set-up): make that first call outside any stream capture.  All calls on a device
 * share the array, which keeps the contents of the last call; the call clears what it
 * needs, but calls whose work overlaps on the GPU (different streams, or different
 * host threads) race and must be serialised by the caller.  Repeated or out-of-range
 * coordinates give NaN energies.  Returns DENSER_ERR_INVALID_ARG, before launching
 * anything, for NULL, host, misaligned or other-device input pointers and for
 * lambda <= 0.  A CUDA runtime error left pending by earlier calls of the process is
 * cleared on entry, so that it is not reported as this call's failure. */
#define DENSER_NOALLOC_MAX_BLOCKS 16384
int denser_energy_noalloc(const int32_t* coords, const float* f, const float* w, const float* u,
                          const float* p, int64_t n_blocks, double lambda, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DENSER_H */
