/*
 * lbm.h -- C ABI of the GB300 (sm_103a) Lagrangian large-deformation lattice
 * Boltzmann solver (Faust, Schlueter, Mueller & Mueller, arXiv 2208.13769).
 *
 * The library advances one 2D plane-strain body (a "context") by the update of
 * Algorithm 1 (Sec. 5): BGK collision with He forcing (Eq. col), streaming
 * (Eq. stream), bounce-back / anti-bounce-back boundary rules (Eqs. bbcon,
 * abbcon, Sec. 6), moments (Eq. moment), the trapezoidal displacement update,
 * H = Grad u (Eq. defgrad), the neo-Hooke first Piola-Kirchhoff stress P(F)
 * of Sec. 7, the Poisson stress Pbar(H) (Eq. Plin) and the source
 * 1S = rho0 b + Div(P + Pbar) (Eq. source1).
 *
 * Conventions shared by every entry point:
 *  - Plain C types only.  Every call returns an lbm_status and never aborts,
 *    prints or throws.  A CUDA error inside a call puts the context in a
 *    sticky error state: later calls on it return LBM_E_CUDA.
 *  - The library owns all device memory of a context (allocated in
 *    lbm_create, freed in lbm_destroy).  Host buffers passed in are only read
 *    (or written, for outputs) during the call; the caller keeps ownership.
 *  - Work is issued on the context's CUDA stream (lbm_desc.cuda_stream, or a
 *    stream the context owns when that is NULL).  lbm_step is asynchronous;
 *    lbm_read_fields and lbm_sync synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Units: any consistent set.  The time step is derived, not passed:
 *    dt = dX / (sqrt(3) C_s), C_s = sqrt(mu / rho0) (Sec. 7's printed time
 *    steps follow this relation).
 *  - Geometry: nx x ny nodes.  Along a bounded axis node k sits at
 *    (k + 1/2) dX and the walls lie half a spacing outside the edge nodes;
 *    along a periodic axis node k sits at k dX.
 *  - Field layout on the host: row-major [ny][nx][ncomp], FP64.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

/* Entry points keep default visibility when the library is built with
 * hidden visibility for everything else. */
#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_E_INVALID = 1,  /* bad argument; nothing was changed */
    LBM_E_OOM = 2,      /* device or host allocation failed */
    LBM_E_CUDA = 3,     /* CUDA runtime error; the context is unusable */
    LBM_E_UNSTABLE = 4, /* a non-finite value or J <= 0 was met (Sec. 7 needs J > 0) */
    LBM_E_TIMEOUT = 5,  /* a bounded device-side wait gave up */
    LBM_E_STATE = 6     /* call out of order (e.g. step before material/boundaries) */
} lbm_status;

/* Storage type of the populations (the arithmetic type follows in brackets):
 * F64 (FP64), F32 (FP32), F16 and BF16 (FP32 arithmetic, populations stored
 * as 16-bit values of f_i / (w_i 2^-s) with a per-context power-of-two scale
 * s; f^eq vanishes at rest, so these are deviations from the rest state). */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 } lbm_storage;

/* Displacement carry: NATIVE keeps u in the arithmetic type; COMPENSATED keeps
 * it as an unevaluated sum of two FP32 numbers (about 48 significant bits),
 * so that Grad u stays accurate when |u| is large; COMPENSATED16 keeps the
 * same sum with the low word stored in 16 bits (FP16 of lo 2^k, k fixed per
 * context from nx, ny and dX so that |u| up to 8 max(nx, ny) dX keeps about
 * 35 significant bits; beyond that the low word saturates and u keeps FP32
 * precision): 12 bytes per node for both components instead of 16.
 * F16/BF16 always use COMPENSATED; F64 always uses FP64. */
typedef enum { LBM_UCARRY_NATIVE = 0, LBM_UCARRY_COMPENSATED = 1, LBM_UCARRY_COMPENSATED16 = 2 } lbm_ucarry;

/* Time level of the source 1S in the moment computation (Sec. 5):
 * EXPLICIT  -- Algorithm 1: the time-t source enters collision and moment
 *              (0: the value of a zeroed lbm_desc, and the Python binding's
 *              default).
 * PREDICTOR -- the predictor-corrector the paper's footnote to Sec. 5 offers:
 *              1S(t+dt) evaluated from the explicitly predicted u*(t+dt)
 *              corrects j and u and is the next collision's source (stable
 *              over more materials: Poisson ratio up to 0.40 in periodic and
 *              Dirichlet bodies, where EXPLICIT needs lambda <= mu).
 * EXTRAPOLATED -- the variant Sec. 5 gives for an O(dt^3) error: 1S(t+dt)
 *              evaluated from the trapezoidal u(t+dt) of j extrapolated
 *              linearly from j(t - dt) and j(t) (j(-dt) = j(0)); as above it
 *              is also the next collision's source.  Stable only for
 *              lambda = mu; two more carry planes (16 B per node update in
 *              FP32); single bodies only (lbm_batch_create rejects it). */
typedef enum { LBM_SCHEME_EXPLICIT = 0, LBM_SCHEME_PREDICTOR = 1, LBM_SCHEME_EXTRAPOLATED = 2 } lbm_scheme;

typedef struct {
    int32_t nx, ny;      /* nodes along x and y; each >= 3 */
    double dX;           /* lattice spacing (> 0) */
    int32_t storage;     /* lbm_storage */
    int32_t u_carry;     /* lbm_ucarry (ignored for F64, F16, BF16) */
    int32_t scheme;      /* lbm_scheme */
    int32_t f16_scale_log2; /* s for F16/BF16 (0 = library default 10) */
    const double* u0;    /* host, [ny][nx][2] initial displacement, NULL = 0 */
    const double* v0;    /* host, [ny][nx][2] initial velocity, NULL = 0 */
    void* cuda_stream;   /* cudaStream_t to issue work on; NULL: the context
                            creates (and destroys) a non-blocking stream of its own */
    int32_t device;      /* CUDA device ordinal */
} lbm_desc;

/* Creates a context: validates desc, allocates the device state and copies u0,
 * v0 to the device.  The populations are initialised lazily, by the first
 * lbm_step or lbm_read_fields after material and boundaries are set
 * (Algorithm 1's initialisation: f_i = f_i^eq(r, j, Pbar) with r = -rho0 Div u0,
 * j = rho0 v0, Pbar = Pbar(Grad u0)).  *out receives the context, or NULL on
 * error.  Errors: LBM_E_INVALID (null pointers, nx or ny < 3, dX <= 0, unknown
 * enum, size overflow: a padded plane of (nx + 168..231) x (ny + 6) nodes must
 * hold fewer than 2^31 elements, e.g. bodies up to about 46 000 x 46 000),
 * LBM_E_OOM, LBM_E_CUDA. */
LBM_API lbm_status lbm_create(const lbm_desc* desc, lbm_ctx** out);

/* Material of Sec. 7 (2D compressible neo-Hooke, plane strain) and the BGK
 * relaxation omega = dt / tau (Eq. col; the paper never fixes tau).
 * body_force: b, per unit mass (NULL = 0).  Requires mu > 0, rho0 > 0,
 * lambda > -mu, 0 < omega < 2; else LBM_E_INVALID.  Only before the first
 * step (afterwards LBM_E_STATE). */
LBM_API lbm_status lbm_set_material(lbm_ctx* ctx, double lambda, double mu, double rho0, double omega,
                            const double body_force[2]);

/* Edge kinds for lbm_set_boundary. */
enum { LBM_PERIODIC = 0, LBM_DIRICHLET = 1, LBM_NEUMANN = 2 };

/* Boundary condition of one edge (Sec. 6).  edge: 0 = x-, 1 = x+, 2 = y-,
 * 3 = y+.  PERIODIC must be set on both edges of an axis.
 * DIRICHLET: prescribed displacement u*(t) = value + rate t, imposed through
 *   bounce-back with the wall momentum j* = rho0 rate (Eq. bbcon).
 * NEUMANN: prescribed first Piola-Kirchhoff traction T*(t): value (T0) before
 *   times[0] and from times[2] on; between, it rises linearly from T0 to
 *   rate (T1) over times[1] (times[1] = 0: a step).  Imposed through
 *   anti-bounce-back with Pbar* (Eq. abbcon, Sec. 6).
 * times may be NULL (0, 0, +inf).  Only before the first step. */
LBM_API lbm_status lbm_set_boundary(lbm_ctx* ctx, int32_t edge, int32_t kind, const double value[2],
                            const double rate[2], const double times[3]);

/* A rectangular hole in the body (Sec. 7's plate with a square hole): the
 * nodes x0 <= x < x1, y0 <= y < y1 (hole = {x0, x1, y0, y1}) are removed.
 * Its faces lie half-way between the body's last node and the first removed
 * one and are Neumann boundaries with a constant traction each: traction
 * holds (Tx, Ty) for the faces at x0, x1, y0, y1 in that order (NULL:
 * traction-free).  A face takes the linear ghost of the differences and
 * anti-bounce-back (Eq. abbcon) with its outward normal (pointing into the
 * hole); a link through a corner of the hole takes both faces, N = (N1 +
 * N2)/sqrt(2), T* = (T1 + T2)/sqrt(2).  Only before the first lbm_step /
 * lbm_read_fields / lbm_diagnostics, after the boundaries of both axes are
 * set.  The hole keeps 4 nodes from bounded edges and 5 from periodic seams
 * (so that its band of boundary nodes clears the body's).  Errors:
 * LBM_E_INVALID (hole out of range or empty, traction not finite),
 * LBM_E_STATE. */
LBM_API lbm_status lbm_set_hole(lbm_ctx* ctx, const int32_t hole[4], const double traction[8]);

/* Advances nsteps (>= 0) time steps (Algorithm 1, one iteration each) on
 * the context's stream, replayed as CUDA graphs of 64 steps for long runs.
 * A step is the fused stream-collide-constitutive update in one launch of
 * the interior kernel and one of the edge tiles on a side stream (or the
 * edge tiles alone for a small body), plus, where the interior kernel runs
 * across a periodic seam (lbm_tuning.plan 2), a launch copying the nodes
 * next to the seam into their periodic images.  The observable fields (u,
 * v, r) are captured at the last step.  Asynchronous.  Errors: LBM_E_STATE (material or boundaries unset),
 * LBM_E_INVALID (nsteps < 0), LBM_E_CUDA. */
LBM_API lbm_status lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Measurement aid (no counterpart in the paper).  Advances `nsteps` time
 * steps exactly as lbm_step does (same kernels, same arithmetic, same
 * results), but launch by launch without graphs, with a CUDA event on the
 * context's stream before and after each of a step's two launches (the
 * interior kernel and the edge-band kernel).  out[0] is the mean duration of
 * the interior launch, out[1] of the edge-band launch, out[2] of their sum,
 * in milliseconds, averaged over all steps but the last (which also writes
 * the read-out fields; with nsteps == 1 it is the only one); out[3] is the
 * number of nodes the interior launch advances (nodes at least 2 from a
 * bounded edge and 3 from a periodic seam).  out[0] and out[3] are 0 for a
 * body too small to have an interior.  Synchronises the stream.
 * Errors: LBM_E_INVALID (nsteps outside 1..4096, out NULL), LBM_E_STATE,
 * LBM_E_OOM, LBM_E_CUDA, and LBM_E_UNSTABLE / LBM_E_TIMEOUT as lbm_sync. */
LBM_API lbm_status lbm_profile_steps(lbm_ctx* ctx, int64_t nsteps, double out[4]);

/* Measurement aid (no counterpart in the paper): the interior kernel alone,
 * `nlaunches` launches back to back on the context's stream between two CUDA
 * events, after one untimed launch; out[0] is the mean duration of a launch
 * in milliseconds, out[1] the number of nodes one launch advances.  The edge
 * bands are not advanced meanwhile, so these launches compute no solution:
 * the state the next step reads (and the device's instability flag) is
 * saved on the device before them and restored after, and the context
 * continues exactly as if the call had not been made.  Allocates a device
 * copy of that state (the population and carry planes of one parity) for
 * the call.  Synchronises.  Errors: LBM_E_INVALID (nlaunches outside
 * 1..4096, out NULL, a body too small to have an interior), LBM_E_STATE,
 * LBM_E_OOM, LBM_E_CUDA. */
LBM_API lbm_status lbm_profile_interior(lbm_ctx* ctx, int64_t nlaunches, double out[2]);

/* Decomposition of the step (no counterpart in the paper; it changes how
 * the work is split, never the result: the interior settings give
 * bit-identical fields; the plan decides which kernel advances the nodes
 * more than two nodes from an edge, whose results agree to rounding).  The
 * interior kernel's row pipeline has a latency floor per launch (about 13 us
 * in FP32 with its shortest 8-row tiles) that small bodies do not fill, while edge tiles
 * take one memory round trip each: below the size thresholds of plan 0 the
 * edge tiles alone are faster (2 to 5 times up to 256 x 256). */
typedef struct {
    int32_t ring_slots; /* rows of the bulk-copy ring, 4..8 (all of them in flight); 0: default (4) */
    int32_t chunk_rows; /* rows per CTA, >= 8; 0: one wave of CTAs over the SMs, at least 8 rows
                           each (default) */
    int32_t aligned;    /* 1: the fewest strips of equal width on 32-byte sector boundaries (at
                           most 120 columns; 112 for 16-bit storage); 2: the same on 16-byte
                           boundaries (at most 124 columns; 120 for 16-bit storage);
                           0: 124-column strips; -1: default (0; in a batch: 0 for 16-bit
                           storage, 1 otherwise) */
    int32_t plan;       /* 0: by size (default): a body of fewer than 2^17 nodes (3 x 2^17 in FP64)
                           runs as small tiles of the edge kernel only, a larger one as the
                           interior kernel plus the edge bands (a 3-node band each side of a
                           periodic seam included); 1: edge tiles only; 2: the interior kernel
                           wherever the body allows it, across periodic seams too (a launch
                           after each step then copies the images of the nodes next to a
                           seam) */
} lbm_tuning;

/* Sets the decomposition; only before the first lbm_step / lbm_read_fields /
 * lbm_diagnostics (LBM_E_STATE after).  Errors: LBM_E_INVALID (out of range). */
LBM_API lbm_status lbm_set_tuning(lbm_ctx* ctx, const lbm_tuning* tuning);

/* The decomposition in use once the context has run (rows per CTA and ring
 * depth as planned), else the one requested. */
LBM_API lbm_status lbm_get_tuning(const lbm_ctx* ctx, lbm_tuning* tuning);

/* Autotuner: times `steps` graph-replayed steps of scratch contexts with
 * desc's size, storage, carry, scheme, stream and device, zero initial
 * fields, lambda = mu = 0.3, and the given edge kinds (periodic edges in
 * pairs), for each candidate decomposition (the interior kernel with ring 4,
 * 5, 6 x rows per CTA one wave, 32, 96, 256 x both strip grids, and edge
 * tiles only), and returns the fastest in *best
 * (its time per step in *best_ms, may be NULL).  The time of a step does not
 * depend on the field values, so the choice holds for any body of that shape.
 * Allocates and frees one scratch context at a time.  Synchronises.
 * Errors: LBM_E_INVALID, and those of lbm_create / lbm_step. */
LBM_API lbm_status lbm_autotune(const lbm_desc* desc, const int32_t edge_kind[4], int64_t steps,
                                lbm_tuning* best, double* best_ms);

/* Field bits for lbm_read_fields; the output holds the requested fields in
 * this bit order, each as [ny][nx][ncomp] FP64. */
enum {
    LBM_FIELD_U = 1,      /* displacement u, 2 comps */
    LBM_FIELD_V = 2,      /* velocity v = j / rho0, 2 comps */
    LBM_FIELD_P = 4,      /* first Piola-Kirchhoff P(Grad u), 4 comps row-major */
    LBM_FIELD_PBAR = 8,   /* Poisson stress Pbar(Grad u), 3 comps (11, 12, 22) */
    LBM_FIELD_R = 16,     /* zeroth moment r = sum_i f_i, 1 comp */
    LBM_FIELD_SIGMA = 32, /* Cauchy stress J^-1 P F^T, 3 comps (11, 12, 22) */
    LBM_FIELD_J = 64      /* J = det F, 1 comp */
};

/* Number of doubles lbm_read_fields writes for mask (0 for an invalid mask). */
LBM_API int64_t lbm_fields_size(const lbm_ctx* ctx, uint32_t mask);

/* Reads fields at the current time t_n = n dt into host memory out
 * (out_len doubles, at least lbm_fields_size).  Stresses are evaluated from
 * u(t_n) with the solver's central differences and ghost rules.  Synchronises
 * the stream.  *t_out (may be NULL) receives t_n.  Returns LBM_E_UNSTABLE if
 * any step so far met a non-finite value or J <= 0 (the fields are still
 * written).  Errors: LBM_E_INVALID (mask, out_len), LBM_E_STATE, LBM_E_CUDA. */
LBM_API lbm_status lbm_read_fields(lbm_ctx* ctx, uint32_t mask, double* out, int64_t out_len,
                           double* t_out);

/* Diagnostics at the current time (deterministic fixed-order reduction):
 * out[0..1] total momentum sum j, out[2] kinetic energy sum |j|^2 / (2 rho0),
 * out[3] strain energy sum W(F) (Sec. 7's W, with ln J), out[4] min J,
 * out[5] 1 if a non-finite value was met else 0 -- all per unit cell volume
 * dX^2 omitted (plain node sums).  Synchronises.  out: 6 host doubles. */
LBM_API lbm_status lbm_diagnostics(lbm_ctx* ctx, double out[6]);

/* Blocks until the context's queued work is done; reports LBM_E_UNSTABLE like
 * lbm_read_fields. */
LBM_API lbm_status lbm_sync(lbm_ctx* ctx);

/* Steps taken so far and the derived time step (NULL pointers allowed). */
LBM_API lbm_status lbm_get_info(const lbm_ctx* ctx, int64_t* steps, double* dt);

/* Bytes of device memory the context holds (the copies of u0 and v0 are
 * released once the initialisation has run), and the algorithmic bytes one
 * node update moves (populations plus carries, read once and written once). */
LBM_API lbm_status lbm_memory_info(const lbm_ctx* ctx, int64_t* device_bytes, int64_t* bytes_per_node_update);

/* Checkpoint and resume (no counterpart in the paper).  The state of a
 * context after its last step, in the library's own layout: the
 * populations, the displacement and source carries (whole planes, with the
 * ghost and image rows and columns), the read-out fields and the step
 * count, behind a header naming the format, size, scheme and time step.
 * lbm_state_size: bytes of a saved state (0 for NULL).
 * lbm_read_state: writes the state into the caller's host buffer `out`
 * (out_len >= lbm_state_size); runs the initialisation first if no step has
 * run; synchronises.  Errors as lbm_read_fields.
 * lbm_write_state: replaces the context's state by a saved one (from a
 * context created with the same size, storage, carry and scheme, and with
 * the same material, hence time step); the boundaries and material must be
 * set, and should be those the state was computed with.  The next lbm_step
 * continues from the saved step exactly as the saved context would have
 * (bit-identical fields).  The caller owns `in`; it is only read during the
 * call, which synchronises.  Errors: LBM_E_INVALID (a header that does not
 * match this context, in_len), LBM_E_STATE, LBM_E_CUDA. */
LBM_API int64_t lbm_state_size(const lbm_ctx* ctx);
LBM_API lbm_status lbm_read_state(lbm_ctx* ctx, void* out, int64_t out_len);
LBM_API lbm_status lbm_write_state(lbm_ctx* ctx, const void* in, int64_t in_len);

/* Frees the context and its device memory (NULL is allowed). */
LBM_API lbm_status lbm_destroy(lbm_ctx* ctx);

/* ------------------------------------------------------------------------
 * Batches: many bodies advanced by shared launches.
 *
 * The method's step (Algorithm 1 with the boundary rules of Sec. 6) applied
 * to several independent bodies at once: each time step is one launch over
 * the interior tiles of every member and one over their edge tiles, so small
 * or uneven bodies share the GPU instead of each paying its own launches;
 * chunks of 64 steps replay as one CUDA graph.  The batch advances every
 * member with the interior kernel where the body allows it (plan 2 of
 * lbm_tuning, unless the member asked for plan 1), through the same
 * arithmetic as a single body: results are bit-identical to lbm_step on a
 * member that runs plan 2; under the default plan a member stepped alone
 * runs edge tiles only (fewer than 2^17 nodes) or gives its periodic seams
 * edge bands, which agree with the interior kernel to rounding.
 */
typedef struct lbm_batch lbm_batch; /* opaque, owned by the library */

/* Groups n existing contexts.  Members must be distinct, on one device, of
 * one storage format and u-carry (scheme EXPLICIT or PREDICTOR, material,
 * boundaries, sizes and step counts may differ), with material and
 * boundaries set; they are
 * initialised here if they were not, and must outlive the batch.
 * cuda_stream: the batch's stream (NULL: the batch owns a non-blocking one);
 * each lbm_batch_step orders itself after work already enqueued on the
 * members' streams and their later work after itself.  Allocates the batch's
 * parameter table and work lists (a few hundred bytes per member and per
 * tile).  Synchronises.  Errors: LBM_E_INVALID (n < 1, NULL or repeated
 * member, mixed devices or formats, a member of scheme EXTRAPOLATED),
 * LBM_E_STATE (a member not ready), LBM_E_OOM, LBM_E_CUDA. */
LBM_API lbm_status lbm_batch_create(lbm_ctx* const* members, int32_t n, void* cuda_stream, lbm_batch** out);

/* lbm_batch_create with a decomposition of the batch's interior tiles (no
 * counterpart in the paper; it changes the split of the work, never the
 * results): tuning->ring_slots, rows of the bulk-copy ring (4..8; 0: 4),
 * tuning->chunk_rows, rows per interior tile (>= 8; 0: about eight waves of
 * resident CTAs over the batch, 32..256 rows), and tuning->aligned, the
 * strip grid of each member (as for lbm_set_tuning; -1: 124-column strips
 * for 16-bit storage, strips on 32-byte sectors otherwise); plan is ignored
 * (each member keeps its own).  NULL: the defaults.
 * Errors as lbm_batch_create, and LBM_E_INVALID for a tuning out of range. */
LBM_API lbm_status lbm_batch_create_tuned(lbm_ctx* const* members, int32_t n, void* cuda_stream,
                                          const lbm_tuning* tuning, lbm_batch** out);

/* Batch autotuner (no counterpart in the paper): builds scratch contexts
 * with the sizes, storage, carry, scheme, device and edge kinds of
 * `members` (zero initial fields, lambda = mu = 0.3), times `steps`
 * graph-replayed steps of a scratch batch of them for each candidate
 * decomposition (ring 4, 5, 6 x rows per tile default, 32, 64, 128, 256 on
 * the format's default strip grid, then the other two strip grids at the
 * best of those) on a stream of its own, and returns the fastest in *best
 * (its time per step in *best_ms, may be NULL).  The time of a step does not depend on the
 * field values, so the choice holds for the members.  The members are not
 * touched.  Holds as much device memory as the members, for the call.
 * Synchronises.  Errors: LBM_E_INVALID (n < 1, NULL member, steps outside
 * 1..100000, best NULL), and those of lbm_create / lbm_batch_create. */
LBM_API lbm_status lbm_batch_autotune(lbm_ctx* const* members, int32_t n, int64_t steps, lbm_tuning* best,
                                      double* best_ms);

/* Advances every member by nsteps time steps (its step count and time too);
 * the last step also refreshes each member's read-out fields, so
 * lbm_read_fields / lbm_diagnostics on a member then see the new state.
 * Asynchronous.  Errors: LBM_E_INVALID (nsteps < 0), LBM_E_STATE (a member
 * was stepped on its own since the batch was made), LBM_E_CUDA. */
LBM_API lbm_status lbm_batch_step(lbm_batch* batch, int64_t nsteps);

/* Synchronises and writes each member's status (as lbm_sync) to status[i]
 * (n entries; may be NULL); returns the first non-OK status, else LBM_OK. */
LBM_API lbm_status lbm_batch_sync(lbm_batch* batch, int32_t* status);

/* Batch time steps taken, and the CTAs of its interior and edge launches. */
LBM_API lbm_status lbm_batch_get_info(const lbm_batch* batch, int64_t* steps, int32_t* interior_ctas,
                                      int32_t* edge_ctas);

/* Frees the batch (not its members; NULL is allowed).  Synchronises. */
LBM_API lbm_status lbm_batch_destroy(lbm_batch* batch);

/* Self-test of the device-side time-out path (no counterpart in the paper).
 * Every wait of the solver's kernels on an mbarrier (the completion of a bulk
 * copy) polls at most a fixed number of times, then records LBM_E_TIMEOUT
 * and lets the kernel return instead of hanging.  This launches one CTA whose
 * barrier can never complete (two arrivals expected, one made) and waits on
 * it with the same bounded wait, `polls` polls at most (1 .. 2^22); on
 * return *timed_out is 1 when the wait gave up, 0 if it completed (which
 * would be a defect).  Nothing faults or hangs; the CUDA context stays usable.
 * Allocates 4 device bytes; synchronises cuda_stream (NULL: legacy stream).
 * Errors: LBM_E_INVALID, LBM_E_OOM, LBM_E_CUDA. */
LBM_API lbm_status lbm_selftest_bounded_wait(uint32_t polls, void* cuda_stream, int32_t* timed_out);

/* ------------------------------------------------------------------------
 * Allocation-free diagnostics (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc -- code running while a CUDA graph
 * is being captured, code confined to a fixed memory pool, or a process whose
 * device allocator belongs to another runtime that forbids side allocations.
 * lbm_diagnostics_noalloc computes the same six numbers as lbm_diagnostics
 * from caller-owned device fields and allocates nothing: its scratch (partial
 * sums of at most 1024 CTAs, 64 KiB) is a static array inside the library,
 * held on every GPU that loads the library until the process exits.
 *
 * fields_dev: device, 5 planes of nx*ny FP64 in row-major [ny][nx] order --
 *   u_x, u_y, v_x, v_y, r (r is not used).
 * geo: body size, spacing, material, and per edge (x-, x+, y-, y+) the kind
 *   and, for Dirichlet edges, the prescribed displacement at the fields' time
 *   (used by the ghost rule of Grad u).
 * out_dev: device, 8 doubles: sum j_x, sum j_y, kinetic energy, strain
 *   energy, min J, non-finite flag, then two zeros.  Written asynchronously on
 *   cuda_stream (NULL: the legacy default stream); read it after the stream
 *   has finished.
 * Limits: nx, ny >= 3 and nx * ny <= LBM_NOALLOC_MAX_NODES; larger bodies,
 *   null pointers, unknown edge kinds or an unpaired periodic edge return
 *   LBM_E_INVALID without launching anything.  The geometry has no hole: for
 *   a body with one (lbm_set_hole) the removed nodes, whatever the fields
 *   hold there, count as nodes of the body, where lbm_diagnostics skips them.
 * The sums equal lbm_diagnostics' to rounding, not bit for bit: the same
 *   kernels run, but above 1024 x 256 nodes the CTAs here stride over more
 *   nodes each, so the order of the additions differs.
 * The first call in each CUDA context of a device looks up the device address
 * of the static array (cudaGetSymbolAddress); make that first call before any
 * stream capture (also again after a device reset, which ends the context).
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and may return wrong sums.  Each call
 * overwrites every partial it reads, so no clearing between calls is needed.
 * Errors: LBM_E_INVALID, LBM_E_CUDA. */
typedef struct {
    int32_t nx, ny;
    double dX, lambda, mu, rho0;
    int32_t edge_kind[4];
    double edge_u[4][2];
} lbm_field_geometry;

#define LBM_NOALLOC_MAX_NODES 2147483647LL

LBM_API lbm_status lbm_diagnostics_noalloc(const lbm_field_geometry* geo, const double* fields_dev,
                                           double* out_dev, void* cuda_stream);

/* Description of the CUDA error that made the context unusable ("none" if
 * there was none).  Static storage; valid for the context's lifetime. */
LBM_API const char* lbm_last_cuda_error(const lbm_ctx* ctx);

/* Static description of a status code. */
LBM_API const char* lbm_status_string(lbm_status status);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
