/*
 * dg.h - C-ABI of the GB300 nonlinear-damage ADER-DG step (libdg).
 *
 * The library advances the 3-D wave equations of a continuum-damage (CDM,
 * Lyakhovsky) rock on a tetrahedral mesh with the explicit ADER discontinuous
 * Galerkin scheme of arXiv 2502.09714:
 *   - governing equations: Sec. 2.1, Eq. "nonlinear damage models" (strain,
 *     velocity, damage alpha) in the conservative form of Eq. "nonlinear hyper
 *     pdes", CDM stress and damage rate of Eq. "cdb-model";
 *   - modal Dubiner DG in space (Eq. "modal dg space"), ADER Taylor expansion in
 *     time (Eq. "eq:taylor_expansion");
 *   - one step = space-time predictor (Appendix A.1, Eqs. "CKIter-ref-matrix",
 *     "CKIter-ref-source"), volume integral (Eq. "3rd term"), Rusanov face flux
 *     from the neighbour trace (Eqs. "rusanov-flux", "2nd term"), pointwise
 *     damage-rate source (Eq. "rhs term"), update (Eq. "time-integrated").
 *
 * Conventions shared by every call:
 *   - All functions return dg_status (DG_OK = 0) and never throw.  On error the
 *     message is available from dg_last_error(ctx) (or dg_last_error(NULL) for
 *     failures before a context exists).
 *   - Host pointers are borrowed for the duration of the call only; the library
 *     copies what it keeps.  The context owns all device memory it allocates.
 *   - Units are SI.  The 10 conservative variables are, in this order,
 *     (eps_xx, eps_yy, eps_zz, eps_xy, eps_yz, eps_zx, v_x, v_y, v_z, alpha) with
 *     tensor (not engineering) shear strains (Eq. "nonlinear hyper pdes").
 *   - Modal coefficients refer to the orthonormal Dubiner basis of the unit
 *     tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1), mapped affinely onto each
 *     element with the element's vertices listed by increasing vertex id
 *     (elem_vid), whatever their order in elem_xyz.  The same map places the
 *     volume and face quadrature nodes, so both elements of a face evaluate
 *     their traces at the same physical points.
 *     Mode order: total degree ascending, then (i,j,k) lexicographic, where mode
 *     (i,j,k) = c * u^i P_i^(0,0)((2xi-u)/u) * w^j P_j^(2i+1,0)((2eta-w)/w)
 *               * P_k^(2i+2j+2,0)(2zeta-1),  u = 1-eta-zeta, w = 1-zeta,
 *     c = sqrt((2i+1)(2i+2j+2)(2i+2j+2k+3)).  L = (N+1)(N+2)(N+3)/6 modes.
 *   - State arrays use the layout q[members][n_elem][10][L] (member, element,
 *     field, mode); with one member this is q[n_elem][10][L].
 *   - Calls are ordered on the context's CUDA stream.  One context per host
 *     thread.  dg_step, dg_get_state* and dg_receivers_read synchronise the
 *     stream before they return; the other calls may return before the device
 *     work they enqueued has finished.
 *   - Device arithmetic is FP32.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;

typedef enum {
  DG_OK = 0,
  DG_E_ARG = 1,            /* invalid argument (NULL pointer, bad size, bad value) */
  DG_E_MESH = 2,           /* invalid mesh: degenerate element, repeated vertex id,
                              face not matched exactly once, bad boundary tag */
  DG_E_ORDER = 3,          /* polynomial degree not compiled into this library */
  DG_E_OOM = 4,            /* device or host allocation failed */
  DG_E_CUDA = 5,           /* a CUDA runtime call failed (message has the CUDA error) */
  DG_E_STATE = 6,          /* call out of sequence (e.g. dg_step before dg_set_material) */
  DG_E_NONFINITE = 7,      /* a NaN/Inf appeared in the state during dg_step */
  DG_E_NONHYPERBOLIC = 8,  /* mu_eff <= 0 or lambda_eff + 2 mu_eff <= 0 in some cell */
  DG_E_OUTSIDE = 9,        /* a source or receiver point lies in no element */
  DG_E_UNSUPPORTED = 10    /* feature not provided by this build (e.g. members > 1) */
} dg_status;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc must
 * return a device pointer aligned to at least 256 bytes, or NULL on failure.
 * NULL in dg_mesh_desc.alloc selects cudaMalloc/cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} dg_allocator;

typedef struct {
  int64_t n_elem;
  const double* elem_xyz;   /* [n_elem][4][3] vertex coordinates of each element.  Periodic
                               images are allowed: an element straddling a periodic wrap lists
                               its unwrapped coordinates. */
  const int64_t* elem_vid;  /* [n_elem][4] global vertex ids; periodically identified vertices
                               share an id.  Two element faces are neighbours iff their vertex-id
                               triples are equal.  The four ids of an element must differ. */
  const int8_t* face_bc;    /* [n_elem][4] tag of the face opposite local vertex f: 0 = interior
                               or periodic (must be matched exactly once), 1 = free surface,
                               2 = absorbing (Appendix A, "Free surface and absorbing boundary
                               conditions"; must belong to this element only).  Boundary fluxes
                               use the effective Lame parameters of the element's cell mean.
                               Any other tag, a tagged face that is shared or an untagged face
                               that is not matched is DG_E_MESH.  NULL = all 0. */
  int order;                /* polynomial degree N (1..5 compiled) */
  int members;              /* ensemble members M >= 1: M copies of the state advance together
                               on the same mesh, each with its own damage parameters (xi0, C_d;
                               see dg_set_material) and its own copy of the sources and
                               receivers; every kernel of a step runs once over all members.
                               n_elem * members < 2^29. */
  double cfl;               /* Courant number of the default time step (see dg_dt) */
  void* cuda_stream;        /* cudaStream_t to order all work on; NULL = legacy default stream */
  const dg_allocator* alloc;/* optional device allocator, NULL = cudaMalloc */
} dg_mesh_desc;

/* Validate the mesh, match faces, build geometry and reference tables, and
 * allocate device memory.  Element orientation is free (either sign of the
 * Jacobian determinant); |det J| must be > 1e-12 * (edge scale)^3.
 * Errors: DG_E_ARG, DG_E_MESH, DG_E_ORDER, DG_E_UNSUPPORTED, DG_E_OOM, DG_E_CUDA.
 * On success *out owns the context (free with dg_destroy). */
dg_status dg_mesh_create(const dg_mesh_desc* desc, dg_ctx** out);

/* Pointwise law of the step: DG_LAW_CDM (default; Eq. "cdb-model"), DG_LAW_IVM
 * (Eq. "ivm-model" with the Murnaghan coefficients l0 = m0 = n0 = 0, effective Lame
 * parameters of Eq. "effective-ivm") or DG_LAW_NLSHEAR, the nonlinear shear law of
 * the 1-D Riemann verification (Sec. 3.1, Eq. "1d Riemann eqs"):
 *     sigma = lambda0 I1 delta + 2 mu0 (1 - beta gamma) eps,  gamma = sqrt(I2 / 2),
 * whose plane shear response is sigma_xy = 2 mu0 (1 - beta eps_xy) eps_xy for
 * eps_xy >= 0; alpha does not evolve, and the predictor and boundary Jacobians use
 * the secant moduli lambda0 and mu0 (1 - beta gamma) at the cell mean.  Changing
 * the law invalidates the material: call dg_set_material again before dg_step.
 * DG_E_ARG for another value. */
enum { DG_LAW_CDM = 0, DG_LAW_IVM = 1, DG_LAW_NLSHEAR = 2 };
dg_status dg_set_rheology(dg_ctx* ctx, int law);

/* Predictor of the step: DG_PREDICTOR_CK (default; the linearised Cauchy-Kovalevskaya
 * procedure of Appendix A.1, Eqs. "CKIter-ref-matrix" and "CKIter-ref-source") or
 * DG_PREDICTOR_PICARD, the discrete Picard iteration Sec. 5.1 proposes in its place:
 * `iterations` (1..16) sweeps that start from the CK coefficients, evaluate the
 * element-local rate -div F(q) + S(q) of the predictor's polynomial at the N + 1
 * time nodes of the step (flux and damage rate projected by the volume rule) and
 * replace D^{j+1} by the j-th Taylor coefficient of the polynomial through those
 * values; each D^o keeps the CK's form (degree N - o for the wave fields, first
 * order for alpha).  It restores order N + 1 on smooth nonlinear solutions, at
 * several times the cost of a step.  Degrees 1..4 (DG_E_ORDER for 5); DG_E_ARG for
 * another kind or iteration count.  The iterations run in the same launch sequence
 * (dg_step and dg_step_noalloc); dg_profile_read counts them under the predictor. */
enum { DG_PREDICTOR_CK = 0, DG_PREDICTOR_PICARD = 1 };
dg_status dg_set_predictor(dg_ctx* ctx, int kind, int iterations);

/* Limit of the bounded waits with which the tensor-core predictor and corrector
 * (degrees 2..4) wait for their matrix products: `polls` polls of the completion
 * barrier per wait (0 .. 2^31 - 1), or the library's default (2^24) for a negative
 * value.  A wait that runs out makes the kernel stop its work, wait (with the
 * default limit) for the products in flight, free its tensor memory and return; the step then
 * returns DG_E_CUDA ("timed out") and the state is left as computed, so the caller
 * restores it with dg_set_state.  A limit of 0 gives up at the first wait, which
 * is how the failure path is tested without any fault.  Not a passage of the
 * paper: the waits belong to this library's kernels.  DG_E_ARG above 2^31 - 1. */
dg_status dg_set_wait_limit(dg_ctx* ctx, int64_t polls);

/* Per-element material [n_elem][6] = (rho, lambda0, mu0, gamma_r, xi0, C_d):
 * density, Lame parameters of the intact rock, damage modulus gamma_r [Pa],
 * damage onset xi0 (Eq. "cdb-model") and damage-rate coefficient C_d [1/(Pa s)].
 * Requires rho > 0, mu0 > 0, lambda0 + 2 mu0 > 0, gamma_r >= 0, C_d >= 0 and
 * finite values (DG_E_ARG otherwise).  member_xi0_cd: NULL (every member takes
 * xi0 and C_d from mat) or [members][n_elem][2] per-member (xi0, C_d), C_d >= 0;
 * non-NULL with one member is DG_E_ARG.  rho, lambda0, mu0 and gamma_r are
 * shared by the members.  Under DG_LAW_IVM the rows are
 * (rho, lambda0, mu0, gamma_b, tau_b, unused) with gamma_b > 0 [Pa] the scale of
 * the storage energy and tau_b > 0 [s] the damage time scale, and
 * member_xi0_cd must be NULL.  Under DG_LAW_NLSHEAR the rows are
 * (rho, lambda0, mu0, beta, unused, unused) with beta >= 0, member_xi0_cd NULL.
 * Also fixes the default time step dt = cfl * min_e 2 r_in(e) / ((2N+1) c_p(e)),
 * r_in the inradius, c_p = sqrt((lambda0 + 2 mu0)/rho). */
dg_status dg_set_material(dg_ctx* ctx, const double* mat, const double* member_xi0_cd);

/* Moment-tensor point sources, replacing any previous set (n = 0 clears).
 * A source acts on the strain equations as the rate
 *     d eps/dt -= C0^{-1} : M * w(t) * delta(x - x_s),
 * C0 the intact isotropic stiffness of the host element, M = m[6] in the field
 * order (Mxx, Myy, Mzz, Mxy, Myz, Mzx).  w(t): stf 0 = Ricker
 * (1 - 2 (pi f0 tau)^2) exp(-(pi f0 tau)^2), tau = t - t0 (M then is the peak
 * moment rate); stf 1 = Gaussian rate of standard deviation f0_or_sigma and unit
 * integral centred at t0 (M the total moment).  Each step adds the exact time
 * integral of w over [t_n, t_n + dt].  The host element is the first element
 * (in input order) whose closure contains x (DG_E_OUTSIDE if none).
 * Requires dg_set_material first (DG_E_STATE). */
typedef struct {
  double x[3];
  double m[6];
  int stf;
  double f0_or_sigma;
  double t0;
} dg_point_source;
dg_status dg_set_source(dg_ctx* ctx, const dg_point_source* src, int64_t n);

/* Set the modal state q[members][n_elem][10][L] (FP64 or FP32 host arrays, or
 * an FP32 device array in the same layout for the _device form) and the time t. */
dg_status dg_set_state(dg_ctx* ctx, const double* q, double t);
dg_status dg_set_state_f32(dg_ctx* ctx, const float* q, double t);
dg_status dg_set_state_device(dg_ctx* ctx, const float* q_dev, double t);

/* Read the modal state into q_out[members][n_elem][10][L] and the time into
 * *t_out (t_out may be NULL). */
dg_status dg_get_state(dg_ctx* ctx, double* q_out, double* t_out);
dg_status dg_get_state_f32(dg_ctx* ctx, float* q_out, double* t_out);
dg_status dg_get_state_device(dg_ctx* ctx, float* q_dev_out, double* t_out);

/* Advance n_steps >= 0 steps of size dt (dt <= 0 selects dg_dt(ctx)).  Each
 * step runs the predictor, the corrector (volume, source, faces, update), the
 * point sources and the receiver sampling on the device.  Reads the device
 * status word once at the end: DG_E_NONFINITE if a NaN/Inf reached the state,
 * DG_E_NONHYPERBOLIC if an effective P or S modulus became non-positive (the
 * state is left as computed; restore it with dg_set_state).  Requires material
 * and state (DG_E_STATE). */
dg_status dg_step(dg_ctx* ctx, int64_t n_steps, double dt);

/* One step from a host state to a host state: q_in and q_out are FP32 host
 * arrays [members][n_elem][10][L] (they may be the same array).  Equivalent to
 * dg_set_state_f32(q_in, current time), dg_step(1, dt), dg_get_state_f32(q_out),
 * with the same arithmetic, but with one member the transfers overlap the
 * step: the elements are cut into chunks, the upload of one chunk runs while the
 * previous one is predicted, the faces run as soon as both their sides are
 * predicted, and the download of one chunk runs while the corrector works on the
 * next (page-locked host arrays are needed for the overlap;
 * pageable ones work without it).  Advances the time by dt.  Requires the
 * material (DG_E_STATE); errors as dg_step. */
dg_status dg_step_host(dg_ctx* ctx, const float* q_in, float* q_out, double dt);

/* The element chunks of dg_step_host with one member, for inspection (host only,
 * no device needed): chunk k holds elements [bounds[k], bounds[k + 1]) of a mesh
 * of n_elem elements.  Every chunk start is a multiple of 16.  Meshes of at most
 * 12,288 elements take chunks of 4096 elements (the last one shorter).  Larger
 * ones take a first chunk of max(4096, n_elem / 16) elements rounded up to 16
 * and a last chunk of that size plus up to 15 (nothing hides these chunks'
 * transfers), with one to seven chunks between, all of one size (a multiple of
 * 16, at least 4096) but the last of them, which is not larger.  Writes the first
 * min(cap, count + 1) entries of bounds and returns the chunk count; -1 for
 * n_elem < 1, cap < 0, or a NULL bounds with cap > 0. */
int dg_host_chunks(int64_t n_elem, int64_t* bounds, int cap);

/* One step that allocates no memory, for callers that cannot call
 * cudaMalloc while they step (a host process under a fixed device-memory
 * budget, code running between the capture of other work, or an embedding
 * that forbids allocation after set-up).  The paper has no counterpart: it is
 * an interface of this library only.
 * q_in and q_out are caller-owned FP32 device arrays in the state layout
 * [n_elem][10][L]; q_out receives the state one step of size dt later
 * (dt <= 0 selects dg_dt(ctx)).  The context's own state, time, sources,
 * receivers and counters are neither read nor changed; point sources are not
 * applied.  The step's intermediate data (converted states, predictor output,
 * cell speeds, face fluxes, status word) live in one file-scope device array of
 * 16 MiB that every GPU loading the library holds until the process exits, so
 * the mesh must satisfy n_elem*(2q + d) + 4*ceil(n_elem/4) + n_faces*f + 64
 * <= 4,194,304 floats with q = 4*ceil(10 L / 4), d the predictor size per
 * element and f = 4*ceil(9 (N+1)^2 / 4), n_faces = interior faces + boundary
 * faces (a mesh without boundary faces has n_faces = 2 n_elem: 2,772 elements
 * at N = 4, 9,868 at N = 2); larger meshes are rejected with DG_E_ARG.
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  Every
 * call reuses the same array, so calls whose work overlaps on the GPU (other
 * streams, other threads, other contexts) race and must be serialised by the
 * caller.  Requires dg_set_material (DG_E_STATE) and one member
 * (DG_E_UNSUPPORTED otherwise).  Status as for dg_step. */
dg_status dg_step_noalloc(dg_ctx* ctx, const float* q_in, float* q_out, double dt);

/* Register R receivers at xyz[R][3] (replaces previous ones, resets traces).
 * After every step the velocity (v_x, v_y, v_z) at each receiver is recorded.
 * DG_E_OUTSIDE if a point lies in no element. */
dg_status dg_receivers(dg_ctx* ctx, const double* xyz, int64_t R);

/* Copy the recorded traces out[n_rec][members][R][3] (n_rec = steps since
 * dg_receivers, at most cap records are copied) and report the number recorded
 * in *n_rec.
 * Traces are kept for at most 65536 steps after dg_receivers. */
dg_status dg_receivers_read(dg_ctx* ctx, float* out, int64_t cap, int64_t* n_rec);

/* Default time step (0 before dg_set_material), current time, sizes. */
double dg_dt(const dg_ctx* ctx);
double dg_time(const dg_ctx* ctx);
int64_t dg_n_modes(int order);

/* Counters since creation: steps taken and kernels launched by dg_step. */
typedef struct {
  int64_t steps;
  int64_t kernel_launches;
  int64_t element_updates;
} dg_stats;
dg_status dg_get_stats(const dg_ctx* ctx, dg_stats* out);

/* Per-kernel timing: when enabled, dg_step records CUDA events around each
 * kernel on the context's stream; dg_profile_read returns, per kernel kind,
 * the number of launches and the summed device milliseconds since the last
 * enable.  Kinds: 0 predictor (with the Picard iterations when they run),
 * 1 corrector (volume terms, face projection and update), 2 point source,
 * 3 receivers, 4 face fluxes. */
typedef struct {
  int64_t launches;
  double total_ms;
} dg_kernel_time;
dg_status dg_profile_enable(dg_ctx* ctx, int on);
dg_status dg_profile_read(dg_ctx* ctx, dg_kernel_time* out, int cap, int* n_kinds);

/* Host-side reference data of degree `order`, for validation without a GPU.
 * which: 0 volume nodes [Nq][4] (xi, eta, zeta, weight, weights sum to 1/6);
 *        1 face nodes [Nf][3] (s, t, weight; weights sum to 1);
 *        2 time nodes [Nt][2] (tau in [0,1], weight; weights sum to 1);
 *        3 basis values at the volume nodes [Nq][L];
 *        4 basis gradients at the volume nodes [Nq][L][3].
 * Writes at most cap doubles; *count receives the number of doubles of the
 * full table.  DG_E_ORDER for an unsupported degree, DG_E_ARG otherwise. */
dg_status dg_reference_table(int order, int which, double* out, int64_t cap, int64_t* count);

/* Gradient of the receiver misfit by the discrete adjoint of the step.
 * Starting from the context's state Q^0 at time t0, n_steps steps of size dt
 * (dt <= 0 selects dg_dt) give the misfit
 *     J = 1/2 sum_{k=1..n_steps} dt sum_r |v_r(Q^k) - ref[k-1][r]|^2,
 * v_r the velocity at receiver r of dg_receivers (FP64 sum).  The call returns
 * J in *misfit and, when the pointers are not NULL, dJ/dxi0 and dJ/dC_d per
 * element (grad_xi0, grad_cd: [n_elem] FP64, the damage onset and rate
 * coefficient of Eq. "cdb-model" in dg_set_material's rows) and dJ/dQ^0
 * (grad_q0: [n_elem][10][L] FP64, the state layout).
 * The gradient is that of the FP32 step the library takes (predictor, face
 * fluxes, corrector, point sources): each product of the step is transposed,
 * including the dependence of the star matrices on the effective Lame
 * parameters of the cell mean (Eq. "effective-cdb") and of the Rusanov speed
 * C = max(cp-, cp+) (Eq. "rusanov-flux") on both cells.  At the non-smooth points
 * the damage rate max(0, .) has derivative zero on its flat side, and a tie of
 * the two P speeds splits the derivative of the max in halves.  The
 * parameter-gradient sums over steps and the misfit are FP64.
 * The step history is kept by binomial checkpointing (revolve): `snapshots`
 * state copies in all (one holds Q^0), so that the forward steps number
 * dg_revolve_cost(n_steps, snapshots) + 1; each adjoint step recomputes its own
 * predictor.  snapshots = 0 takes as many copies as 80 % of the free device
 * memory holds beside the call's other buffers, at most n_steps + 1 (the whole
 * history, one forward sweep) and at most 4096.  ref: host FP32 [n_steps][R][3], R receivers.  The context's state,
 * time and recorded traces are left unchanged.  info: NULL or the counts and
 * device milliseconds of the forward steps, the adjoint steps (predictor
 * recompute, adjoint kernels and misfit terms) and the snapshot copies.
 * Free-surface and absorbing faces are differentiated too (their flux through
 * the own trace and the effective Lame parameters of the cell mean).
 * Requires the CDM law, the CK predictor, one member (DG_E_UNSUPPORTED
 * otherwise), material, state and at least one receiver
 * (DG_E_STATE); DG_E_ARG for n_steps outside 1..2^20, snapshots outside
 * 0..4096 or a plan of more than 2^27 forward steps; DG_E_OOM if the
 * snapshots (snapshots x n_elem x 4 ceil(10 L / 4) floats) do not fit;
 * DG_E_NONFINITE / DG_E_NONHYPERBOLIC as dg_step. */
typedef struct {
  int64_t forward_steps;
  int64_t adjoint_steps;
  double forward_ms;
  double adjoint_ms;
  double copy_ms;
} dg_adjoint_info;
dg_status dg_adjoint_gradient(dg_ctx* ctx, int64_t n_steps, double dt, const float* ref, int snapshots,
                              double* misfit, double* grad_xi0, double* grad_cd, double* grad_q0,
                              dg_adjoint_info* info);

/* The binomial checkpointing plan behind dg_adjoint_gradient, for inspection
 * (host only, no device needed).  Reversing n_steps steps with `snapshots`
 * state slots (slot 0 holds the initial state) takes
 *     T = t n - C(s + 1 + t, t - 1)  forward steps,  s = snapshots - 1,
 * t the least integer with C(s + 1 + t, t) >= n (T = n (n - 1) / 2 for s = 0);
 * dg_revolve_cost returns T (-1 for bad arguments).  dg_revolve_plan writes
 * *forward_steps = T and up to cap actions as triples (kind, a, b): kind 0
 * advance the current state from step a to step b, 1 store the current state
 * (step b) in slot a, 2 restore slot a (step b), 3 the adjoint of step a; the
 * full count goes to *n_actions.  DG_E_ARG for n_steps outside 1..2^20,
 * snapshots outside 1..4096 or T > 2^27. */
dg_status dg_revolve_plan(int64_t n_steps, int snapshots, int64_t* forward_steps, int64_t* actions,
                          int64_t cap, int64_t* n_actions);
int64_t dg_revolve_cost(int64_t n_steps, int snapshots);

const char* dg_last_error(const dg_ctx* ctx);
void dg_destroy(dg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DG_H */
