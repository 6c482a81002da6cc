/*
 * qhd.h -- C ABI of the GB300 QHD split-operator simulator.
 *
 * The library evolves the Quantum Hamiltonian Descent Schroedinger equation
 *
 *     i d psi/dt = [ e^{phi_t} (-1/2 Lap) + e^{chi_t} f(x) ] psi
 *
 * (Leng, Hickman, Li, Wu, "Quantum Hamiltonian Descent", arXiv 2303.01471,
 * Eq. (main1) / Eq. (qhd_operator)) on the regular periodic mesh of a box
 * [lo, hi]^d with N_d = 2^q points per axis (Sec. "Implementing QHD using
 * product formulae", "Spatial discretization", Eq. (wave-rep)).  Time stepping
 * is the pseudo-spectral product formula of Eqs. (prod_qhd), (prod_qhd_fft)
 * and Algorithm 1 in its symmetric (Strang) form: per step a potential half
 * phase, a forward FFT along every axis, the kinetic phase diagonal in Fourier
 * space, an inverse FFT and a second potential half phase, with both schedule
 * coefficients taken at the step midpoint.  Observables follow Eq. (expect_O)
 * and the success criterion of the Fig. 2 caption.
 *
 * Further families in this header: the spectrum of H(t) (qhd_apply_hamiltonian,
 * qhd_lowest_eigenpairs), the tensor-core DFT form (qhd_set_transform), the
 * learned surrogate (qhd_fno_*), QHD on the finite-difference box mesh of the
 * analog implementation (qhd_lattice_*, its own context and fixed-point state).
 *
 * Conventions shared by every entry point (the box mesh states its own state
 * format)
 * ---------------------------------------
 * - Arrays are row-major with the LAST axis fastest.  The grid point with
 *   multi-index (j_0, ..., j_{d-1}) sits at x_k = lo[k] + j_k (hi[k]-lo[k]) / n[k].
 * - psi is complex64: interleaved (re, im) float32 pairs, batch * G values,
 *   G = prod n[k]; instance b occupies [b*G, (b+1)*G).  The caller owns it.
 * - Device memory (psi, workspace) and the CUDA stream belong to the caller.
 *   The library allocates no device memory: everything it needs lives in the
 *   caller's workspace of qhd_workspace_bytes() bytes (256-byte aligned).
 * - All work is enqueued on the caller's stream.  qhd_set_potential*,
 *   qhd_observables and qhd_destroy synchronise that stream; the other calls
 *   only enqueue.
 * - Every call returns a qhd_status; no exception crosses the ABI.  A failed
 *   argument check leaves the context unchanged (except a rejected potential,
 *   which discards the previous one).  A CUDA error or a device
 *   time-out makes the context sticky-failed: later calls return the same
 *   status until qhd_destroy.  qhd_last_error() gives the message.
 * - One context must not be used from two host threads at once.
 */
#ifndef QHD_H
#define QHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qhd_ctx qhd_ctx; /* opaque; created by qhd_init_grid, freed by qhd_destroy */

typedef enum {
    QHD_OK = 0,
    QHD_ERR_INVALID_ARG = 1, /* a pointer, size or value is out of its documented range */
    QHD_ERR_UNSUPPORTED = 2, /* valid request the library does not implement           */
    QHD_ERR_STATE = 3,       /* call order violated (e.g. evolve before set_potential)  */
    QHD_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed (sticky)    */
    QHD_ERR_TIMEOUT = 5,     /* a bounded device wait gave up (sticky)                  */
    QHD_ERR_WORKSPACE = 6    /* workspace NULL, too small or misaligned                 */
} qhd_status;

/* Damping schedule families (Eq. (qhd_operator) leaves phi_t, chi_t free). */
typedef enum {
    /* e^{phi_t} = c_phi / (eps + t^3), e^{chi_t} = c_chi t^3.  With c_phi = 2,
     * eps = s = 1e-3, c_chi = 2 this is Eq. (nonconvex_QHD_h) of the paper's
     * simulations; c_chi = 2 sigma scales the potential weight. */
    QHD_SCHED_NESTEROV = 0,
    /* phi(t), chi(t) piecewise linear through n_samples points (t strictly
     * increasing), constant outside [t[0], t[n-1]]; a = e^phi, b = e^chi. */
    QHD_SCHED_TABLE = 1,
    /* e^{phi_t} = c_phi / (eps + |t|^{p+1}), e^{chi_t} = c_chi |t|^{2p-1},
     * p = power in [0.5, 8].  The three-parameter Hamiltonian of
     * Eq. (qhd_operator_convex) with the ideal scaling condition
     * (Eq. (ideal_scaling)) met with equality, alpha_t = log p - log t,
     * beta_t = p log t + log C, gamma_t = p log t, has e^{alpha-gamma} =
     * p t^{-(p+1)} and e^{alpha+beta+gamma} = p C t^{2p-1}: c_phi = p,
     * c_chi = p C, with eps regularising t -> 0.  p = 2 is QHD_SCHED_NESTEROV. */
    QHD_SCHED_POWER = 2
} qhd_sched_kind;

typedef struct {
    int32_t kind;       /* qhd_sched_kind                                        */
    double c_phi;       /* NESTEROV, POWER: > 0                                   */
    double eps;         /* NESTEROV, POWER: >= 0; eps = 0 is allowed only if no   */
                        /*           step midpoint is t = 0                       */
    double c_chi;       /* NESTEROV, POWER: >= 0                                  */
    const double *t;    /* TABLE: host arrays of n_samples values, copied by the  */
    const double *phi;  /*        library during qhd_set_schedule                 */
    const double *chi;
    int64_t n_samples;  /* TABLE: 1 .. 256                                        */
    double power;       /* POWER: p in [0.5, 8]; ignored by the other kinds       */
} qhd_schedule;

/* Observables of one instance (Eq. (expect_O); Fig. 2 caption). */
typedef struct {
    double t;          /* current simulation time                                   */
    double norm;       /* sum_x |psi_x|^2  (l2 norm of Eq. (wave-rep); 1 ideally)   */
    double e_f;        /* E[f] = sum_x |psi_x|^2 f(x)  (FP64 f, FP64 accumulation)  */
    double p_succ;     /* sum of |psi_x|^2 over mesh points with |x - x*|_2 < radius */
                       /* (Euclidean on the box, not periodic)                      */
    double x_star[3];  /* grid minimiser of f (lowest flat index on ties); 0 beyond d */
    int64_t steps_done;/* Strang steps taken since the last qhd_reset_state          */
} qhd_obs;

/* Bytes of device workspace a context for this grid and batch needs.
 * Returns 0 for an unsupported shape (see qhd_init_grid). */
size_t qhd_workspace_bytes(int ndim, const int64_t *n, int64_t batch);

/*
 * Create a context.  ndim in 1..3; every n[k] a power of two in 2..1024;
 * lo[k] < hi[k], both finite; 1 <= batch <= 65535 independent instances
 * sharing the mesh (each with its own f and schedule); G <= 2^30 and
 * batch * G <= 2^34.  psi_dev: caller-owned device
 * buffer of batch*G complex64, 16-byte aligned (the passes move two points per
 * 16-byte copy; an 8-byte aligned pointer is refused with
 * QHD_ERR_INVALID_ARG).  work_dev: caller-owned device
 * buffer of work_bytes >= qhd_workspace_bytes(...), 256-byte aligned.
 * stream: a cudaStream_t (NULL = legacy default stream).  Both buffers must
 * outlive the context.  *out is set only on QHD_OK.
 */
qhd_status qhd_init_grid(qhd_ctx **out, int ndim, const int64_t *n, const double *lo,
                         const double *hi, int64_t batch, void *psi_dev, void *work_dev,
                         size_t work_bytes, void *stream);

/*
 * Load the objective sampled on the mesh (the diagonal potential operator V of
 * Algorithm 1):
 * f_host is host FP64, batch*G values in psi's layout.  Copies f into the
 * workspace (FP64 for E[f], plus a 32-bit fixed-point copy with a per-instance
 * power-of-two scale used for the potential phase), finds the grid minimiser x*.
 * Every value must be finite and max f - min f < 2^31 per instance, else
 * QHD_ERR_INVALID_ARG and the previous potential is discarded (evolve and
 * observables return QHD_ERR_STATE until a valid one is loaded).
 * Synchronises the stream.
 */
qhd_status qhd_set_potential(qhd_ctx *ctx, const double *f_host);

/* Same as qhd_set_potential with f already in device memory (FP64, batch*G). */
qhd_status qhd_set_potential_device(qhd_ctx *ctx, const double *f_dev);

/*
 * Set the damping schedule: s points to batch schedules (one per instance).
 * TABLE samples are copied.  Invalid parameters give QHD_ERR_INVALID_ARG.
 */
qhd_status qhd_set_schedule(qhd_ctx *ctx, const qhd_schedule *s);

/* psi <- G^{-1/2} in every instance (the uniform superposition that Algorithm 1
 * and Eq. (prod_qhd) start from),
 * t <- 0, steps_done <- 0.  Enqueued on the stream. */
qhd_status qhd_reset_state(qhd_ctx *ctx);

/* Set the simulation time without touching psi (psi is the caller's buffer and
 * may be written directly, e.g. to resume from a checkpoint). */
qhd_status qhd_set_time(qhd_ctx *ctx, double t);
qhd_status qhd_get_time(const qhd_ctx *ctx, double *t_out, int64_t *steps_done_out);

/*
 * Advance every instance by n = round(T/dt) Strang steps (Eq. (prod_qhd_fft)
 * with the symmetric split): step j uses a = e^{phi}, b = e^{chi} at
 * t_{j+1/2} = t + (j + 1/2) dt.  T/dt must be a positive integer to within
 * 1e-9 relative; dt finite and nonzero (dt < 0 with T < 0 runs time backwards,
 * exactly undoing a forward run up to rounding).  Requires set_potential and
 * set_schedule.  Enqueued on the stream (asynchronous); t <- t + n dt.
 */
qhd_status qhd_evolve(qhd_ctx *ctx, double T, double dt);

/*
 * Trajectory of the observables (the loss E[f](t) of Eq. (expect_O) and the
 * success probability of the Fig. 2 caption along the evolution): advances by
 * n = round(T/dt) steps like qhd_evolve and, after every `every` steps, writes
 * (sum |psi|^2, E[f], P_succ) of every instance into traj_dev, a caller-owned
 * device array of (n/every) * batch * 3 doubles: point k, instance b at
 * traj_dev[(k*batch + b)*3 + 0..2].  every >= 1 must divide n.  Asynchronous
 * on the stream (no host synchronisation between points).
 */
qhd_status qhd_evolve_trajectory(qhd_ctx *ctx, double T, double dt, int64_t every, double radius,
                                 double *traj_dev);

/*
 * Time-stepping formula used by qhd_evolve (default QHD_SPLIT_STRANG).
 * QHD_SPLIT_STRANG: P(dt/2) F^-1 K(dt) F P(dt/2) with a, b at the step midpoint
 *   (second order).
 * QHD_SPLIT_LIE_TROTTER: the first-order product formula exactly as printed in
 *   Eq. (prod_qhd) / Algorithm 1: psi_{j+1} = F^-1 K(dt a_j) F P(dt b_j) psi_j with
 *   a_j = e^{phi(t_j)}, b_j = e^{chi(t_j)}, t_j = t + j dt (left end point).
 * Unknown kinds give QHD_ERR_INVALID_ARG.  Applies to later qhd_evolve calls.
 */
enum { QHD_SPLIT_STRANG = 0, QHD_SPLIT_LIE_TROTTER = 1 };
qhd_status qhd_set_splitting(qhd_ctx *ctx, int kind);

/*
 * Discretisation of the kinetic operator -Lap/2 used by later qhd_evolve
 * calls (default QHD_KINETIC_SPECTRAL).
 * QHD_KINETIC_SPECTRAL: exact on the mesh's Fourier modes, eigenvalue
 *   |k|^2 / 2 with k_d = 2 pi m_d / L_d (Eq. (prod_qhd_fft)).
 * QHD_KINETIC_FD2: the central second difference of Eq. (discretize-pde),
 *   (2 psi_j - psi_{j+1} - psi_{j-1}) / (2 h_d^2) per axis with h_d = L_d / N_d,
 *   on the same periodic mesh (the paper states it with vanishing boundary
 *   values; the periodic wrap is kept here so that the same transforms
 *   diagonalise it); eigenvalue (2 / h_d^2) sin^2(pi m_d / N_d) per axis.
 * Every transform path (FFT passes and the tensor-core form) honours it.
 * Unknown kinds give QHD_ERR_INVALID_ARG.
 */
enum { QHD_KINETIC_SPECTRAL = 0, QHD_KINETIC_FD2 = 1 };
qhd_status qhd_set_kinetic(qhd_ctx *ctx, int kind);

/*
 * Transform used by qhd_evolve for the per-axis DFTs of the kinetic step
 * (Eq. prod_qhd_fft).  QHD_TRANSFORM_FFT (default): the shared-memory FFT
 * passes.  QHD_TRANSFORM_TC_DFT: each axis transform is a dense product with
 * the n x n DFT matrix on the tensor cores (this library's tcgen05 GEMM: FP16
 * operands, every 16-term MMA sum exact in FP32 and added to the result with
 * round-to-nearest; the phases, transposes and operand splits run in this
 * library's kernels, with the same fixed-point phase arguments as the FFT
 * path).  products selects the operand form:
 *   3: block-scaled hi/lo -- each 16 consecutive values of a row share a
 *      power-of-two exponent and are cut into two FP16 integer slices (21
 *      bits below the block maximum), the DFT matrix into two (21 bits);
 *      three slice products.  The DFT matrix's last slice is re-rounded every
 *      step with a pseudo-random offset (floor(r + u), u in [0, 1) per step),
 *      so its rounding is exact on average over steps instead of a fixed
 *      perturbation repeated in every transform;
 *   5: as 3 with the DFT matrix in three slices (32 bits) and two more
 *      products;
 *  10: fixed-point slices on a per-instance power-of-two scale (data to 2^-28
 *      of the instance maximum, DFT matrix 29 bits) whose slice-level sums
 *      are integers the FP32 accumulator holds exactly (n <= 512).
 * Neither form lets the tensor cores round a partial sum, so neither drifts.
 *
 * Requires ndim == 2 and n[0] == n[1], a power of two in 64..1024 (64..512 for
 * products = 10), and batch <= 65535 (else QHD_ERR_UNSUPPORTED;
 * qhd_tc_workspace_bytes returns 0 for these and for other products).
 * tc_work_dev: caller-owned device buffer, 256-byte aligned, of at least
 * qhd_tc_workspace_bytes(...) bytes, kept until the transform is changed or
 * the context destroyed (else QHD_ERR_WORKSPACE); it holds the DFT matrices
 * (and, for 3 and 5 products, their last slice before rounding in FP32), the
 * FP16 operands, the block exponents and the FP32 products.  No device
 * memory is allocated.  transform = QHD_TRANSFORM_FFT releases the
 * tensor-core state and ignores the other arguments.  Unknown transforms or
 * products other than 3, 5 and 10 give QHD_ERR_INVALID_ARG.  Synchronises the
 * stream (uploads the DFT matrices).
 */
enum { QHD_TRANSFORM_FFT = 0, QHD_TRANSFORM_TC_DFT = 1 };
size_t qhd_tc_workspace_bytes(int ndim, const int64_t *n, int64_t batch, int products);
qhd_status qhd_set_transform(qhd_ctx *ctx, int transform, int products, void *tc_work_dev,
                             size_t tc_work_bytes);

/* Library (cuBLAS) GEMM calls this context has issued so far: always 0, the
 * tensor-core transform runs on this library's own GEMM kernel. */
int64_t qhd_library_call_count(const qhd_ctx *ctx);

/* CTAs per instance (2-D grids held in one thread-block cluster for a whole
 * chunk of steps) or per plane (3-D plane passes) of the cluster engine; 0 for
 * the generic passes or a NULL context.  For 2-D grids whose axis 0 has 64 or
 * 128 points, a batch with at most (SM count / wide split) instances runs on
 * twice the default CTAs per instance (4 for 64, 8 for 128: half the rows per
 * CTA), fixed at qhd_init_grid.  A batched group (qhd_group_*) uses the same
 * split by default. */
int qhd_cluster_ctas(const qhd_ctx *ctx);

/*
 * Observables of every instance: out_host[batch] receives qhd_obs; prob_dev
 * (optional, NULL to skip) receives |psi|^2 as float32, batch*G values.
 * radius > 0 (the paper's success radius is 0.1).  Synchronises the stream.
 */
qhd_status qhd_observables(qhd_ctx *ctx, qhd_obs *out_host, float *prob_dev, double radius);

/*
 * qhd_observables_static -- observables of states the caller already holds,
 * with no context, no workspace and no device allocation.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc where they
 * need the observables: e.g. an application whose device memory is entirely
 * reserved by another allocator, where one more allocation would fail or
 * fragment that pool, or a latency-critical caller that must not pay for
 * cudaMalloc, which can synchronise the device.
 *
 * The reduction scratch is a fixed array of QHD_STATIC_SCRATCH_BYTES inside the
 * library; every GPU that loads the library holds that much memory until the
 * process exits.  Limits: batch <= 32 instances, every n[k] a power of two in
 * 2..1024, ndim 1..3.  Larger requests return QHD_ERR_INVALID_ARG.
 *
 * Inputs (device pointers on the current device): psi_dev, batch*G complex64
 * in the layout of qhd_init_grid; f_dev, batch*G FP64 objective values.
 * x_star: host array of batch*3 doubles, the minimiser coordinates used for
 * the success probability (entries beyond ndim ignored).  radius > 0.
 * Outputs: out_dev, a device array of batch*3 doubles receiving per instance
 * (sum |psi|^2, sum |psi|^2 f, sum of |psi|^2 within radius of x_star), the
 * same quantities and accumulation order as qhd_observables; prob_dev
 * (optional, NULL to skip) receives |psi|^2 as float32.  Everything is
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream); the
 * call does not synchronise.
 *
 * The first call on a device looks up the device address of the scratch
 * array with that device current; make that first call before any stream
 * capture.  All calls share the one array and each call overwrites every part
 * of it it reads, so nothing needs clearing, but calls whose work overlaps on
 * the GPU (e.g. on two streams, or from two host threads) race on it.
 */
#define QHD_STATIC_SCRATCH_BYTES (1u << 20)
qhd_status qhd_observables_static(int ndim, const int64_t *n, const double *lo, const double *hi,
                                  int64_t batch, const void *psi_dev, const double *f_dev,
                                  const double *x_star, double radius, double *out_dev,
                                  float *prob_dev, void *stream);

/* Kernel launches this context has issued so far (for launch accounting). */
int64_t qhd_launch_count(const qhd_ctx *ctx);

/*
 * Device-time accounting per kernel class (instrumentation; the paper has no
 * counterpart).  qhd_timing_enable(ctx, every) with every > 0 makes
 * qhd_evolve record a CUDA event pair on the stream around every launch that
 * belongs to a step j with j % every == 0 (and around the prep launch of
 * every chunk); every = 0 turns it off.  At most 65536 pairs are kept until
 * read.  qhd_timing_read synchronises on the recorded events and writes, per
 * class, the summed device milliseconds and the number of timed launches
 * into arrays of QHD_KCLASS_COUNT entries (either may be NULL), then forgets
 * the records if reset != 0.
 */
enum {
    QHD_KCLASS_PREP = 0,       /* schedule + phase tables of a chunk              */
    QHD_KCLASS_ROW = 1,        /* fastest-axis pass with the potential phase      */
    QHD_KCLASS_AXIS1_FWD = 2,  /* 3-D: forward transform along axis 1             */
    QHD_KCLASS_AXIS0 = 3,      /* axis-0 pass: forward, kinetic phase, inverse    */
    QHD_KCLASS_AXIS1_INV = 4,  /* 3-D: inverse transform along axis 1             */
    QHD_KCLASS_ONED = 5,       /* 1-D: all steps of a chunk in one launch         */
    QHD_KCLASS_PLANE = 6,      /* 3-D: cluster pass over axes 1 and 2 with the    */
                               /*      potential phase                           */
    QHD_KCLASS_WHOLE = 7,      /* 2-D: all steps of a chunk, instance resident in */
                               /*      one thread-block cluster                   */
    QHD_KCLASS_TC_SPLIT = 8,   /* tensor-core transform: phase / transpose and    */
                               /*      FP16 split kernels                         */
    QHD_KCLASS_TC_GEMM = 9,    /* tensor-core transform: tcgen05 GEMM launches    */
    QHD_KCLASS_COUNT = 10
};
qhd_status qhd_timing_enable(qhd_ctx *ctx, int every);
qhd_status qhd_timing_read(qhd_ctx *ctx, double *ms_out, int64_t *launches_out, int reset);

/*
 * Spectrum of the QHD Hamiltonian (the probability spectrum and energy ratio
 * of the paper's section on the three phases of QHD):
 *   H(t) = e^{phi_t} (-Lap/2) + e^{chi_t} f
 * on the context's mesh, with its kinetic discretisation (qhd_set_kinetic)
 * and instance `inst`'s f and schedule.  H is real symmetric on the mesh.
 *
 * qhd_apply_hamiltonian: out = H(t) in for one instance; in_dev, out_dev are
 *   G complex64 values each (distinct buffers).  Asynchronous on the stream.
 *   Kinetic part by the context's transforms (forward along every axis, the
 *   real factor e^{phi} |k|^2 / 2 or its finite-difference counterpart, inverse),
 *   potential part e^{chi} f in as a pointwise product.
 * qhd_lowest_eigenpairs: m Lanczos steps with full reorthogonalisation from a
 *   seeded random start vector, then the k lowest Ritz pairs (1 <= k <= m,
 *   2 <= m <= 1024, m <= G).  Convergence of the low levels needs m of order
 *   sqrt(spread of H / level gap): a few hundred on meshes of 64^2 and up (the
 *   returned residuals show it).  Outputs (host arrays of k doubles, each optional):
 *   eigvals (ascending), residuals ||H u - theta u|| with ||u|| = 1 (computed
 *   with qhd_apply_hamiltonian), overlaps |<u, psi>|^2 / <psi, psi> with the
 *   instance's current state (the probability spectrum); eigvecs_dev
 *   (optional, k * G complex64) receives the normalised Ritz vectors.  A
 *   single start vector resolves each distinct eigenvalue once: a degenerate
 *   level may appear only once.  work_dev: caller-owned, 256-byte aligned,
 *   qhd_spectrum_workspace_bytes(ctx, m) bytes.  Synchronises the stream.
 * Errors: QHD_ERR_STATE without potential and schedule, QHD_ERR_INVALID_ARG
 *   for inst, m, k out of range, QHD_ERR_WORKSPACE for a short workspace.
 */
size_t qhd_spectrum_workspace_bytes(const qhd_ctx *ctx, int m);
qhd_status qhd_apply_hamiltonian(qhd_ctx *ctx, int64_t inst, double t, const void *in_dev, void *out_dev);
qhd_status qhd_lowest_eigenpairs(qhd_ctx *ctx, int64_t inst, double t, int m, int k, uint64_t seed,
                                 void *work_dev, size_t work_bytes, double *eigvals, double *residuals,
                                 double *overlaps, void *eigvecs_dev);

/*
 * Learned surrogate: a Fourier neural operator (FNO) that maps an instance's
 * sampled objective f on an n x n mesh of [0,1]^2 and its schedule scale sigma
 * to a predicted |psi(T)|^2 (a distribution over the mesh), trained on
 * distributions this library's solver computes.  The paper has no surrogate;
 * the solver stays the reference and the fallback.  Network per instance:
 * features ((f - mean f)/std f, sigma, x0, x1) -> lift to `width` channels ->
 * `layers` Fourier layers a = SC(v) + W v + b, v' = gelu(a) (no gelu after the
 * last), SC a spectral convolution over the modes kx in {0..modes-1} U
 * {n-modes..n-1}, ky in {0..modes-1} with complex width x width weights per
 * mode -> h = gelu(Wp1 v + bp1) (`hidden` channels) -> z = Wp2 h + bp2 ->
 * p = softmax of z over the mesh.  Loss: KL(p_true || p) averaged over the
 * batch.  Every step runs in this library's kernels; activations are BF16
 * (act_bf16 = 1) or FP32 (0, for gradient checks), arithmetic and
 * accumulation FP32, weights FP32.
 *
 * Parameters: one caller-owned FP32 device vector of qhd_fno_param_count(cfg)
 * values (8-byte aligned), laid out as lift W[width][4], b[width]; per layer
 * R[2 modes][modes][width][width] complex (re, im pairs), W[width][width],
 * b[width]; then Wp1[hidden][width], bp1[hidden], Wp2[hidden], bp2; each block
 * starts at an even offset.  Gradients use the same layout.  Limits: n a power
 * of two in 8..256, width even in 2..32, 1 <= modes, 2 modes <= n, layers
 * 1..8, hidden even in 2..128, batch_max <= 65535; else the size queries
 * return 0 and create returns QHD_ERR_INVALID_ARG.  The workspace
 * (caller-owned, 256-byte aligned, qhd_fno_workspace_bytes) holds the
 * activations of batch_max instances and, with train != 0, the backward
 * buffers and the Adam moments (zeroed at create).  All calls are asynchronous
 * on `stream` except qhd_fno_loss_grad with a non-NULL loss_host, which
 * synchronises to return the loss.
 *
 * qhd_fno_forward: f_dev = batch x n x n FP64 (row-major per instance),
 *   sigma_dev = batch FP32, p_dev = batch x n x n FP32 output.
 * qhd_fno_loss_grad: forward + backward against p_true_dev (batch x n x n
 *   FP32 distributions); grad_dev (param_count FP32) is overwritten with
 *   dL/dparams; QHD_ERR_STATE without training buffers.
 * qhd_fno_adam_step: params -= lr * mhat / (sqrt(vhat) + eps), step t >= 1.
 */
typedef struct qhd_fno qhd_fno;
typedef struct {
    int32_t n, width, modes, layers, hidden, act_bf16;
} qhd_fno_config;
int64_t qhd_fno_param_count(const qhd_fno_config *cfg);
size_t qhd_fno_workspace_bytes(const qhd_fno_config *cfg, int64_t batch_max, int train);
qhd_status qhd_fno_create(qhd_fno **out, const qhd_fno_config *cfg, int64_t batch_max, int train,
                          float *params_dev, void *work_dev, size_t work_bytes, void *stream);
qhd_status qhd_fno_forward(qhd_fno *fno, const double *f_dev, const float *sigma_dev, int64_t batch,
                           float *p_dev);
qhd_status qhd_fno_loss_grad(qhd_fno *fno, const double *f_dev, const float *sigma_dev,
                             const float *p_true_dev, int64_t batch, float *grad_dev, double *loss_host);
qhd_status qhd_fno_adam_step(qhd_fno *fno, const float *grad_dev, float lr, float beta1, float beta2,
                             float eps, int64_t t);
int64_t qhd_fno_launch_count(const qhd_fno *fno);
const char *qhd_fno_last_error(const qhd_fno *fno);
qhd_status qhd_fno_destroy(qhd_fno *fno);

/*
 * QHD on the finite-difference box mesh (the paper's section on implementing
 * QHD on quantum Ising machines: Eq. (discretize-pde), Eq. (finite-qhd-discrete)
 * and the relaxed form Eq. (relaxed-qhd-discrete) with Eq. (relaxed_adjacency);
 * its classical simulation is the Sim-QHD solver of the QP benchmark).  The
 * mesh has r cells per edge of [0,1]^d: points x_j = j / r, j = 0..r, so
 * n = r + 1 per axis and G = n^d; arrays are row-major, last axis fastest.
 *
 *     H(t) = e^{phi_t} sum_k K_k + e^{chi_t} F,     K = -(r^2 / 2) A  (per axis)
 *
 * A is the chain adjacency (QHD_LATTICE_CHAIN: the central second difference
 * with vanishing values beyond the mesh, its -2 diagonal dropped as a global
 * phase as the paper does) or the relaxed A' with the entries
 * sqrt((j+1)(r-j)/r), j = 0..r-1 (QHD_LATTICE_RELAXED: S_x / sqrt(r) on the
 * Hamming-weight states of r qubits, the operator the Hamming encoding
 * realises).  Time stepping: the Strang product formula with a = e^{phi},
 * b = e^{chi} at the step midpoints.  The axis terms commute, so the kinetic
 * factor exp(-i dt a sum_k K_k) is applied as the dense n x n matrix
 * exp(-i dt a K) along every axis; the potential phase exp(-i theta F) uses the
 * exact fixed-point turns of the Fourier-mesh path.  The state is held in
 * fixed point: every amplitude component is an int32 in units of 2^-29, each
 * line product is an exact int64 sum rounded once, so the norm stays within a
 * few 1e-7 over 10^3 steps however concentrated the state is.
 *
 * Limits: ndim 1..6, r 1..16, 1 <= batch <= 65535, batch * G <= 2^31.  Device memory
 * and the stream belong to the caller; ownership, asynchrony, error statuses
 * and sticky CUDA failures follow the qhd_ctx conventions above.
 *
 * qhd_lattice_workspace_bytes: bytes of 256-byte aligned device workspace;
 *   0 for sizes out of the limits.
 * qhd_lattice_init: psi_dev caller-owned, 8-byte aligned, batch*G pairs of
 *   int32 (re, im) in units of 2^-29: the working state, read and written by
 *   the library (use qhd_lattice_get_state / _set_state for complex64); kind a
 *   qhd_lattice_kind; work_dev / work_bytes as sized above; stream a
 *   cudaStream_t (0 = legacy default stream).
 * qhd_lattice_get_state: out_dev (batch*G complex64, 8-byte aligned) receives
 *   the state.  Async.
 * qhd_lattice_set_state: the state from in_dev (batch*G complex64), rounded to
 *   the nearest 2^-29.  Every instance must have norm^2 <= 1 + 1e-3 (the
 *   integer line products are sized for it) and finite components; otherwise
 *   the state is set to 0 and the call returns QHD_ERR_INVALID_ARG.
 *   Synchronises the stream.
 * qhd_lattice_set_potential: f_dev = batch*G FP64 on the device (copied);
 *   non-finite values or a range >= 2^31 give QHD_ERR_INVALID_ARG and discard
 *   the previous potential.  Synchronises the stream.
 * qhd_lattice_set_qp: F(x) = 1/2 x^T Q x + b^T x on the mesh
 *   (Eq. (finite-quadratic-obj)), formed on the device in FP64 from host arrays
 *   Q_host (batch*d*d, row-major per instance; only its symmetric part enters)
 *   and b_host (batch*d).  Synchronises the stream.
 * qhd_lattice_set_schedule: as qhd_set_schedule (batch schedules).
 * qhd_lattice_reset_state: init = QHD_LATTICE_INIT_UNIFORM (G^{-1/2}) or
 *   QHD_LATTICE_INIT_GROUND (the product over the axes of the ground state of
 *   -A: the amplitudes sqrt(binom(r,j) / 2^r) for A', the Hamming encoding's
 *   initial state; sqrt(2/(r+2)) sin(pi (j+1)/(r+2)) for the chain); t = 0.
 * qhd_lattice_evolve: round(T/dt) Strang steps from the current time, same
 *   rules as qhd_evolve (dt != 0, T/dt an integer within 1e-9, T and dt of
 *   one sign); needs potential and schedule (else QHD_ERR_STATE).  Async.
 * qhd_lattice_observables: out (host, batch): norm, E[f], p_succ (mass within
 *   `radius`, Euclidean, of the mesh argmin x*, lowest flat index on ties),
 *   p_gap (mass on points with f - min f <= gap); prob_dev (optional,
 *   batch*G FP32) receives |psi|^2; marginals_host (optional, batch*d*n
 *   doubles, [b][k][j]) the probabilities of the measurement elements
 *   E^{(k)}_j of Eq. (Ekj).  FP64 accumulation in a fixed order.
 *   Synchronises the stream.
 * qhd_lattice_evolve_trajectory: advances like qhd_lattice_evolve and, after
 *   every `every` steps (every >= 1 dividing round(T/dt)), writes (norm, E[F],
 *   p_succ, p_gap) of every instance into traj_dev, a caller-owned device array
 *   of (n/every) * batch * 4 doubles: point k, instance b at
 *   traj_dev[(k*batch + b)*4 + 0..3].  Asynchronous (no host synchronisation
 *   between points).
 * qhd_lattice_timing_enable / _read: as qhd_timing_* with the kernel classes
 *   QHD_LKCLASS_* (every = 0 switches sampling off).
 */
typedef struct qhd_lattice qhd_lattice;
typedef enum { QHD_LATTICE_CHAIN = 0, QHD_LATTICE_RELAXED = 1 } qhd_lattice_kind;
typedef enum { QHD_LATTICE_INIT_UNIFORM = 0, QHD_LATTICE_INIT_GROUND = 1 } qhd_lattice_init_kind;
enum {
    QHD_LKCLASS_PREP = 0,  /* schedule, potential coefficients, axis propagators */
    QHD_LKCLASS_PASS0 = 1, /* the pass with the potential phase (last axes)      */
    QHD_LKCLASS_PASS1 = 2, /* the other passes                                   */
    QHD_LKCLASS_COUNT = 3
};
typedef struct {
    double t, norm, e_f, p_succ, p_gap;
    double f_min;        /* min of F over the mesh                       */
    int64_t argmin;      /* its flat index (lowest on ties)              */
    int64_t steps_done;  /* steps since the last qhd_lattice_reset_state */
} qhd_lattice_obs;
size_t qhd_lattice_workspace_bytes(int ndim, int r, int64_t batch);
qhd_status qhd_lattice_init(qhd_lattice **out, int ndim, int r, int kind, int64_t batch, void *psi_dev,
                            void *work_dev, size_t work_bytes, void *stream);
qhd_status qhd_lattice_set_potential(qhd_lattice *lat, const double *f_dev);
qhd_status qhd_lattice_set_qp(qhd_lattice *lat, const double *Q_host, const double *b_host);
qhd_status qhd_lattice_set_schedule(qhd_lattice *lat, const qhd_schedule *s);
qhd_status qhd_lattice_reset_state(qhd_lattice *lat, int init);
qhd_status qhd_lattice_get_state(qhd_lattice *lat, void *out_dev);
qhd_status qhd_lattice_set_state(qhd_lattice *lat, const void *in_dev);
qhd_status qhd_lattice_evolve(qhd_lattice *lat, double T, double dt);
qhd_status qhd_lattice_evolve_trajectory(qhd_lattice *lat, double T, double dt, int64_t every, double radius,
                                         double gap, double *traj_dev);
qhd_status qhd_lattice_observables(qhd_lattice *lat, qhd_lattice_obs *out, float *prob_dev, double *marginals_host,
                                   double radius, double gap);
qhd_status qhd_lattice_timing_enable(qhd_lattice *lat, int every);
qhd_status qhd_lattice_timing_read(qhd_lattice *lat, double *ms_out, int64_t *launches_out, int reset);
int64_t qhd_lattice_launch_count(const qhd_lattice *lat);
const char *qhd_lattice_last_error(const qhd_lattice *lat);
qhd_status qhd_lattice_destroy(qhd_lattice *lat);


/*
 * Batched persistent launch over several contexts (no counterpart in the
 * paper; it runs many independent instances of Algorithm 1 at once).
 *
 * A group binds 1..8 contexts that are 2-D with a square mesh of edge 64, 128
 * or 256, use the FFT transform and share one stream, and have a potential and
 * a schedule loaded.  qhd_group_evolve(g, T, dt) evolves every instance of
 * every context by T (the same as qhd_evolve on each context, including its
 * splitting, kinetic operator and clock) in ONE launch per chunk of <= 1024
 * steps: a grid of clusters of 8 CTAs pulls work items from a device queue,
 * first the step tables of each context, then groups of instances, each
 * instance held in the shared memory of `sub` CTAs of a cluster (8 / sub
 * instances per cluster item).  The launch sequence is captured once into a
 * CUDA graph and replayed while T, dt and the contexts' clocks at the call
 * repeat (e.g. reset_state, group_evolve, observables, ...); a change
 * re-captures.  Waits for the tables are bounded: qhd_group_status
 * synchronises the stream and returns QHD_ERR_TIMEOUT if one gave up, which
 * also makes the group and its contexts sticky-failed.
 *
 * cfg (may be NULL for the defaults, every field 0): sub_cluster[k] = CTAs per
 * instance for edge 64 (k = 0: 2, 4 or 8), 128 (k = 1: 4 or 8), 256 (k = 2: 8);
 * min_blocks = resident CTAs per SM the kernel is compiled for (1 or 2);
 * clusters = persistent clusters launched (0: as many as fit at once).  These
 * are the choices the benchmark's autotuner searches.
 *
 * Workspace: caller-owned device memory of qhd_group_workspace_bytes(n_ctx)
 * bytes, 256-byte aligned, kept until qhd_group_destroy.  The contexts must
 * outlive the group.  Errors: QHD_ERR_INVALID_ARG (NULL, duplicate context,
 * contexts on different streams, bad cfg), QHD_ERR_STATE (a context without
 * potential or schedule, or in a failed state), QHD_ERR_UNSUPPORTED (mesh not
 * square 64/128/256, not 2-D, or the tensor-core transform; more than 16 table
 * chunks in one call), QHD_ERR_WORKSPACE, QHD_ERR_CUDA.  evolve only enqueues.
 */
typedef struct qhd_group qhd_group;
typedef struct {
    int32_t sub_cluster[3];
    int32_t min_blocks;
    int32_t clusters;
} qhd_group_config;
size_t qhd_group_workspace_bytes(int n_ctx);
qhd_status qhd_group_create(qhd_group **out, qhd_ctx *const *ctxs, int n_ctx, const qhd_group_config *cfg,
                            void *work_dev, size_t work_bytes);
qhd_status qhd_group_evolve(qhd_group *g, double T, double dt);
qhd_status qhd_group_status(qhd_group *g);
/* Test hook: with on != 0 every later launch waits for one table arrival more
 * than any producer makes, so its waits run out and qhd_group_status reports
 * QHD_ERR_TIMEOUT (a bounded wait giving up; nothing faults). */
qhd_status qhd_group_inject_wait_timeout(qhd_group *g, int on);
/* out (8 values): clusters launched, min_blocks, shared memory per CTA (bytes),
 * kernel launches so far, graph captures so far, CTAs per instance for edge 64,
 * 128, 256 (0 when no context has that edge). */
qhd_status qhd_group_info(const qhd_group *g, int64_t *out);
const char *qhd_group_last_error(const qhd_group *g); /* "" if none; g may be NULL */
qhd_status qhd_group_destroy(qhd_group *g);

/* Dense FP16 product on the 5th-generation tensor cores: the GEMM of the
 * tensor-core transform (qhd_set_transform), exposed for testing and reuse; no
 * counterpart in the paper.  C = alpha * A . B^T + beta * C with A row-major
 * [rows][k] and B row-major [n_cols][k] (FP16, K contiguous, device memory) and
 * C row-major FP32 [rows][ldc] (device).  group_every_mma = 1: every K = 16
 * step accumulates into a fresh tensor-memory partial that is added to the FP32
 * result with a round-to-nearest FMA (when the operands are integers whose
 * 16-term sums stay below 2^24, every partial is exact and the result is the
 * exact sum rounded to nearest at each addition); 2: the same, for floating
 * operands: each MMA truncates its exact sum towards zero to FP32, losing on
 * average the fraction kappa = 2^-24 / (2 ln 2) of it, and the result is scaled
 * by (1 + kappa) to undo that expected loss; 0: one accumulation over all of K
 * in tensor memory (the hardware's accumulation; 128 x 256 tiles when n_cols
 * is a multiple of 256, each finished tile added to C in place).  Requirements: rows >= 1,
 * n_cols a multiple of 128, k of 64, k <= 2^20, ldc >= n_cols and a
 * multiple of 4, 16-byte aligned pointers.  err_dev: 2 device words, zero on
 * entry; word 0 becomes 1 if a bounded wait gave up (~2 s).  Enqueued on
 * stream (a cudaStream_t, NULL = legacy default); nothing is allocated.
 * Errors: QHD_ERR_INVALID_ARG, QHD_ERR_CUDA (launch failure). */
qhd_status qhd_tc_gemm_f16(const void *A_dev, const void *B_dev, float *C_dev, int64_t ldc, int64_t rows,
                           int64_t n_cols, int64_t k, int group_every_mma, float alpha, float beta,
                           unsigned *err_dev, void *stream);
/* Message of the CUDA runtime for the calling thread's last qhd_tc_gemm_f16 ("" after success). */
const char *qhd_tc_gemm_last_error(void);

/* Failure injection for tests of the error contract above (no counterpart in
 * the paper).  With kind = QHD_ERR_CUDA or QHD_ERR_TIMEOUT, the after-th
 * checked CUDA call of this context from now on (a kernel launch, a copy or a
 * stream synchronisation, counted across entry points, after >= 1) is not
 * issued: the entry point that reaches it fails with `kind` exactly as if the
 * runtime had reported an error or a bounded device wait had given up, so the
 * context becomes sticky-failed and every later call except qhd_destroy
 * returns `kind`.  Work enqueued before that call stays enqueued; nothing
 * reaches the GPU in a failed state.  kind = QHD_OK cancels a pending
 * injection.  Errors: QHD_ERR_INVALID_ARG for another kind or after < 1; a
 * context that is already sticky-failed returns its status. */
qhd_status qhd_inject_failure(qhd_ctx *ctx, int kind, int64_t after);

/* Synchronise the stream and free the host-side context (never the caller's
 * buffers).  NULL is accepted. */
qhd_status qhd_destroy(qhd_ctx *ctx);

const char *qhd_status_string(qhd_status s);
const char *qhd_last_error(const qhd_ctx *ctx); /* "" if none; ctx may be NULL */

#ifdef __cplusplus
}
#endif
#endif /* QHD_H */
