/*
 * smap.h -- C ABI of the GB300 Stein-MAP-Seq library (libsmap.so).
 *
 * Stein-MAP-Seq (Seo & Kia, arXiv 2312.08684) estimates the MAP state sequence
 * x_{0:T} of a state-space model from observations z_{1:T} (Section II,
 * Eq. MAP_est). At every step t it moves N particles with L iterations of Stein
 * variational gradient descent toward p(z_t, x_t | previous particle set)
 * (Algorithm 1; directions Eq. SVGD_initial_newupdate for t = 1 and
 * Eq. SVGD_newupdate for t >= 2), then runs one step of a Viterbi max-plus
 * recursion over consecutive particle sets (Eq. forward_recursion); the MAP
 * path is read back by backtracking (Section IV-B, Algorithm 2).
 *
 * Conventions that hold for every call:
 *   - Every call returns an smap_status; nothing throws across the ABI.
 *   - A handle owns all of its device memory (allocated in smap_create, freed in
 *     smap_destroy). The caller owns every buffer it passes in.
 *   - "on_device" = 1 means the data pointers of that call are device pointers
 *     (e.g. torch.Tensor.data_ptr() of a CUDA tensor); 0 means host pointers.
 *   - Work is queued on the handle's stream (smap_config.stream; NULL = the
 *     legacy default stream). Calls that return results to host memory, and
 *     smap_map_sequence / smap_run_batch / smap_viterbi, synchronise that stream
 *     before returning.
 *   - The first CUDA error puts the handle into a failed state: later calls
 *     return SMAP_E_STATE. smap_last_error() gives the message.
 *   - One handle is used by one host thread at a time.
 *   - Arrays are dense, row-major, without padding; d = state dimension,
 *     dy = observation dimension of the model (smap_dims).
 *   - Particles are FP32; cumulative Viterbi scores phi_t and J are FP64.
 */
#ifndef SMAP_H
#define SMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMAP_OK = 0,
    SMAP_E_INVAL = 1,        /* bad argument (size, model parameters, null pointer) */
    SMAP_E_NOMEM = 2,        /* device or host allocation failed */
    SMAP_E_CUDA = 3,         /* a CUDA runtime call failed */
    SMAP_E_STATE = 4,        /* handle already failed, or call out of order */
    SMAP_E_TIMEOUT = 5,      /* a bounded device wait ran out */
    SMAP_E_NONFINITE = 6,    /* a particle or observation became NaN/Inf */
    SMAP_E_UNSUPPORTED = 7   /* valid request the library does not implement */
} smap_status;

/* Compiled-in scenario models. Parameter vectors (FP64), d and dy:
 *  SMAP_MODEL_NGM1D        [a, b, c, omega, t_off, q, r, hcoef]        d=1, dy=1
 *      x_t = a x + b x/(1+x^2) + c cos(omega (t + t_off)) + N(0, q)
 *      z_t = hcoef x_t^2 + N(0, r)          (Section V-A form)
 *  SMAP_MODEL_RANGE_CV2D   [dt, q0, q1, q2, q3, r, nb, b0x, b0y, ...]  d=4, dy=nb (1..8)
 *      state (px, py, vx, vy), constant velocity with step dt, Q = diag(q0..q3);
 *      z_l = ||(px,py) - b_l|| + N(0, r); a NaN entry of z means beacon l was
 *      not heard at that step (Section V-C form)
 *  SMAP_MODEL_CLUTTER_CV2D [dt, q0, q1, q2, q3, r, M, beta, area]      d=4, dy=2M (M 1..32)
 *      constant velocity; z = M points; p(z|x) = (1-beta)(1/M) sum_m
 *      N(z_m; (px,py), r I) + beta/area   (unknown association with outliers,
 *      Section V-B form)
 *  SMAP_MODEL_PLANAR_ARM   [dt, nl, r, q_0..q_{2nl-1}, len_0..len_{nl-1}] d=2nl, dy=2
 *      state (angles, rates), angles += dt * rates; z = sum_l len_l (cos th_l,
 *      sin th_l), th_l = sum_{m<=l} angle_m, noise N(0, r I) (Section V-D form;
 *      the library is compiled for nl = 7)
 *  SMAP_MODEL_LINEAR_GAUSS [dt, q0, q1, q2, q3, r]                     d=4, dy=2
 *      constant velocity, z = (px, py) + N(0, r I)
 *  SMAP_MODEL_RANGE_ZV2D   [q0, q1, r, nb, a0x, a0y, ...]               d=2, dy=nb (1..8)
 *      state (px, py) without a motion prior: x_t = x_{t-1} + N(0, diag(q0, q1));
 *      z_l = ||x - a_l|| + N(0, r), NaN = anchor l not heard (Section V-C's
 *      zero-velocity model)
 *  SMAP_MODEL_SE2_RB       [dt, q0, q1, q2, rr, rb, v, w, nl, L0x, L0y, ...] d=3, dy=2 (nl 1..8)
 *      pose (px, py, th) on SE(2) under constant controls: th' = th + w dt,
 *      (px, py)' = (px, py) + v dt (cos th', sin th') + N(0, diag(q0..q2));
 *      z = (range, bearing) from one of nl landmarks, association unknown:
 *      p(z|x) = (1/nl) sum_l N(zr; ||p - L_l||, rr) N(wrap(zb - b_l); 0, rb),
 *      b_l = atan2(py - L_ly, px - L_lx), wrap into [-pi, pi]; a NaN range means
 *      no measurement at that step (Section V-B's model)
 */
typedef enum {
    SMAP_MODEL_NGM1D = 1,
    SMAP_MODEL_RANGE_CV2D = 2,
    SMAP_MODEL_CLUTTER_CV2D = 3,
    SMAP_MODEL_PLANAR_ARM = 4,
    SMAP_MODEL_LINEAR_GAUSS = 5,
    SMAP_MODEL_RANGE_ZV2D = 6,
    SMAP_MODEL_SE2_RB = 7
} smap_model;

/* Kernel bandwidth h of kappa(x,x') = exp(-||x-x'||^2 / h) (the RBF kernel of
 * Section V, median heuristic of the Table Ex6 caption):
 *   MEDIAN_ITER  h = bw_value * med / log N, med = median of the squared
 *                pairwise distances (i < k; mean of the two middle values when
 *                their count is even), recomputed every SVGD iteration;
 *   MEDIAN_STEP  the same, computed at the first iteration of each step;
 *   FIXED        h = bw_value.
 * N = 1 or med = 0 gives h = 1. */
typedef enum { SMAP_BW_MEDIAN_ITER = 0, SMAP_BW_MEDIAN_STEP = 1, SMAP_BW_FIXED = 2 } smap_bw_rule;

/* Prior term of the direction of Eq. SVGD_newupdate:
 *   MIXTURE   score of log (1/N) sum_j p(x | x_{t-1}^j) (responsibility-weighted)
 *   MEANGRAD  mean over j of grad log p(x | x_{t-1}^j) = Q^-1 (mean_j f_j - x)
 *   MAPCOND   conditioned on the previous MAP estimates (Section V-C): the
 *             score of max_j [phi_{t-1}(j) + log p(x | x_{t-1}^j)], i.e.
 *             Q^-1 (f_{j*} - x) for the maximising predecessor j* (chosen in
 *             FP32, lowest j on ties)
 * They coincide when the previous set has one particle (t = 1). */
typedef enum { SMAP_PRIOR_MIXTURE = 0, SMAP_PRIOR_MEANGRAD = 1, SMAP_PRIOR_MAPCOND = 2 } smap_prior;

/* Stein kernel k(x, x') of the SVGD direction (Eq. svgd_iterate), u = r^2 / h
 * with r = |x - x'| and h the bandwidth of smap_bw_rule:
 *   RBF        exp(-u)                            (the method's kernel, Section V)
 *   IMQ        (1 + u)^(-1/2)                     (Gorham & Mackey 2017)
 *   MATERN32   (1 + s) exp(-s), s = sqrt(3 u)     (Matern nu = 3/2, length sqrt(h))
 * IMQ and Matern are the alternatives of the kernel ablation (Table Ex6). */
typedef enum { SMAP_KERNEL_RBF = 0, SMAP_KERNEL_IMQ = 1, SMAP_KERNEL_MATERN32 = 2 } smap_kernel;

typedef struct smap_handle smap_handle;

typedef struct {
    int model;              /* smap_model */
    const double* params;   /* host, copied at create */
    int n_params;
    int N;                  /* particles per sequence (maximum if N varies), 1..4096 */
    int L;                  /* SVGD iterations per step, >= 0 */
    double step;            /* SVGD step size epsilon (Algorithm 1) */
    int bw_rule;            /* smap_bw_rule */
    double bw_value;        /* scale for the median rules, h for FIXED */
    int prior;              /* smap_prior */
    uint64_t seed;          /* key of the Philox-4x32-10 noise of the particle initialisation */
    int batch;              /* number of independent sequences B >= 1 */
    int max_T;              /* longest sequence the handle can hold */
    const double* x0;       /* host [batch][d]: the known initial states x_0^true */
    void* stream;           /* cudaStream_t the handle works on; NULL: the handle creates its own */
    int kernel;             /* smap_kernel (0 = RBF) */
} smap_config;

/* Validates cfg, allocates the handle's device buffers (particle history
 * [B][max_T][N][d] FP32, backpointers [B][max_T][N] uint16, scores [B][N]
 * FP64, work queue and scratch). No kernel runs. *out is NULL on failure;
 * a failed allocation returns SMAP_E_NOMEM and frees what was allocated.
 * (For tests, the environment variable SMAP_FAIL_ALLOC=k makes the k-th
 * device allocation of a call fail that way.) The library marks the host
 * phases of its entry points with NVTX ranges named after them. */
smap_status smap_create(const smap_config* cfg, smap_handle** out);

/* Frees everything the handle owns (synchronises its stream). NULL is a no-op. */
void smap_destroy(smap_handle* h);

/* d and dy of the handle's model. */
smap_status smap_dims(const smap_handle* h, int* d, int* dy);

/* Back to t = 0 for every sequence; x0 (host [B][d]) replaces the initial
 * states when not NULL. */
smap_status smap_reset(smap_handle* h, const double* x0);

/* Sets the particle count of each sequence (host [B], 1..N); NULL = all N.
 * Only allowed at t = 0 (after create / reset). */
smap_status smap_set_particle_counts(smap_handle* h, const int* N_per_seq);

/* One online step t -> t+1 of Algorithm 2 for every sequence whose active flag
 * is set (active: host [B] bytes, or NULL = all): SVGD on the new particle set
 * (L iterations), then phi_{t+1}, psi_{t+1}. y: [B][dy] FP32 observations z_{t+1}
 * (host or device per on_device). One fused kernel launch; asynchronous. */
smap_status smap_step(smap_handle* h, const float* y, const uint8_t* active, int on_device);

/* Backtracking (Section IV-B) for every sequence at its current length T_s:
 * path [B][max_T+1][d] FP32 (row 0 = x_0^true, rows t > T_s = NaN), J [B]
 * FP64 = phi_{T_s}(i_{T_s}) (either may be NULL). Synchronises the stream. */
smap_status smap_map_sequence(smap_handle* h, float* path, double* J, int on_device);

/* The whole batch from t = 0 in one persistent launch (sequences pulled from
 * a device work queue, longest first), followed by backtracking; the device
 * work is replayed from a CUDA graph after the first call.
 * y_all [B][max_T][dy] FP32; T_per_seq host [B] (1..max_T, NULL = max_T);
 * N_per_seq host [B] (1..N, NULL = N); path / J as in smap_map_sequence.
 * Afterwards the handle holds the final state (smap_get_history etc.). */
smap_status smap_run_batch(smap_handle* h, const float* y_all, const int* T_per_seq,
                           const int* N_per_seq, float* path, double* J, int on_device);

/* Copies of the handle's state: particle sets hist [B][max_T][N][d] FP32 (the
 * final particles of each step), backpointers psi [B][max_T][N] (psi_1 = 0),
 * current scores phi [B][N] FP64, current step counts t [B]. */
smap_status smap_get_history(smap_handle* h, float* hist, int on_device);
smap_status smap_get_backpointers(smap_handle* h, uint16_t* psi, int on_device);
smap_status smap_get_scores(smap_handle* h, double* phi, int on_device);
smap_status smap_get_steps(smap_handle* h, int* t_per_seq);

/* The dynamic programme alone (Eq. forward_recursion + backtracking) over
 * given particle sets hist [B][max_T][N][d] FP32 and observations y_all
 * [B][max_T][dy]: the second stage of Algorithm 2 on fixed supports.
 * T_per_seq / N_per_seq as in smap_run_batch; outputs path / J (may be NULL)
 * and psi [B][max_T][N] (may be NULL). Uses and overwrites the handle's
 * history, score and backpointer buffers. Synchronises the stream. */
smap_status smap_viterbi(smap_handle* h, const float* hist, const float* y_all,
                         const int* T_per_seq, const int* N_per_seq, float* path,
                         double* J, uint16_t* psi, int on_device);

/* Checkpoint and resume of the online state (not in the paper): the known
 * x_0, every sequence's step count, particle count, length and status, the
 * current scores phi_t [B][N], the median guesses of the bandwidth rule, and
 * each sequence's particle sets and backpointer rows up to its current step.
 * smap_state_size gives the bytes smap_save writes now (it grows with the
 * step counts). smap_save copies the state into host memory `buf` of at
 * least that size (synchronises the stream; the handle is not changed).
 * smap_load restores it into a handle created with the same configuration
 * (model, parameters, N, L, step, bandwidth rule and value, prior, kernel,
 * seed, batch, max_T): SMAP_E_INVAL if the configuration or the sizes do not
 * match. After smap_load, smap_step continues exactly as the saved handle
 * would have (same bits). An attached proposal is not part of the state
 * (smap_proposal_get_weights / set_weights save and restore it). */
smap_status smap_state_size(const smap_handle* h, size_t* bytes);
smap_status smap_save(smap_handle* h, void* buf, size_t bytes);
smap_status smap_load(smap_handle* h, const void* buf, size_t bytes);

/* PF-MAP-Seq, the particle-filter comparison method of Section V (Godsill,
 * Doucet and West 2001): for every sequence a bootstrap particle filter with
 * stratified resampling at every step supplies the supports, then the same
 * forward recursion and backtracking as Stein-MAP-Seq give the MAP sequence
 * over them. Per step t: x_1^i = f_1(x_0) + sqrt(q) (.) xi_i; for t >= 2 the
 * step t-1 weights w_j = p(z_{t-1} | x_{t-1}^j) are normalised and summed,
 * u_i = (i + U_i) / N, ancestor a_i = the first j whose cumulative weight
 * exceeds u_i, x_t^i = f_t(x_{t-1}^{a_i}) + sqrt(q) (.) xi_i. xi and U come
 * from Philox-4x32-10 keyed by smap_config.seed (counters (i, t, seq, block)
 * and (i, t, seq, 256)); the filter runs in FP64, the recursion on FP32 copies.
 * Uses the handle's model, N (up to 4096), B, max_T and seed; L, step, the
 * bandwidth, prior, kernel and any attached proposal are ignored. y_all,
 * T_per_seq, N_per_seq, path, J as in smap_run_batch; afterwards the handle
 * holds the filter's particle sets as its history (smap_get_history) and the
 * backpointers (smap_get_backpointers). The first call allocates 8 B N (d + 1)
 * bytes of device memory per sequence (SMAP_E_NOMEM if that fails).
 * Synchronises the stream. */
smap_status smap_pf_run_batch(smap_handle* h, const float* y_all, const int* T_per_seq,
                              const int* N_per_seq, float* path, double* J, int on_device);

/* smap_viterbi for callers that cannot allocate device memory. (The paper has
 * no counterpart; it exists for the library's callers.) Some callers cannot
 * call cudaMalloc: a plug-in whose host application owns the device-memory
 * budget and passes it only input and output buffers, or a control loop that
 * must not enter the allocator while it runs. A handle allocates, so this
 * call takes no handle and allocates nothing.
 *   model / params / n_params  as in smap_config (params: host memory);
 *   x0 [B][d] FP64, hist [B][T][N][d] FP32, y [B][T][dy] FP32: device inputs;
 *   path [B][T+1][d] FP32, J [B] FP64: device outputs (as in smap_viterbi).
 * Its working state (scores, backpointers, transition means, queue, status,
 * backtracking chain) lives in one static 16 MiB device array of the library,
 * which every GPU that loads the library holds until the process exits. Sizes
 * whose working state exceeds 16 MiB (about 2 B T N bytes of backpointers
 * plus 8 B N (2 + d) bytes of scores and means) are rejected with
 * SMAP_E_INVAL and a message on stderr. The first call on a device looks up
 * the array's device address (set-up, once per device, with that device
 * current; done again in the new context after a device reset); make that
 * first call before any stream capture. The call is
 * asynchronous on `stream` (cudaStream_t, NULL = legacy default stream) and
 * clears what it needs at the start of each call; every call shares the
 * array, so calls that overlap on the GPU (other streams or host threads)
 * race. A sequence whose scores become non-finite gets J = NaN. */
smap_status smap_viterbi_noalloc(int model, const double* params, int n_params, int B, int N, int T,
                                 const double* x0, const float* hist, const float* y, float* path,
                                 double* J, void* stream);

/* ---------------------------------------------------------------------------
 * Learned proposal. (Not in the paper: a transport map that replaces most of
 * the SVGD iterations of a step.) A 3-layer perceptron, features -> 256 ->
 * 256 -> d with GELU, BF16 weights and activations on the tensor cores, FP32
 * accumulation, maps a propagated particle u = f_t(x_{t-1}^i) + Q^{1/2} xi
 * (the plain initialisation) and the observation z_t to the displacement that
 * plain SVGD applies to it; the learned step then starts from u + MLP(u, z_t)
 * and runs a few SVGD iterations. Features (at most 32 per row, zero padded),
 * each list ending with the likelihood score g = grad_u log p(z_t | u):
 *   PLANAR_ARM   [u, z, z - h(u), g of the angles]
 *   CLUTTER_CV2D [velocity, the M points relative to the position, nearest first, g of the position]
 *   others       [u, z (unheard = 0), heard flags, g]
 * Training data rows are [32] FP32 features and [16] FP32 displacement targets
 * (zero padded). Parameters: FP32 master vector, padded layout W1 [256][32],
 * b1 [256], W2 [256][256], b2 [256], W3 [16][256], b3 [16]; normalisation
 * vector mu_in [32], sd_in [32], mu_out [16], sd_out [16] (inputs and targets
 * are standardised with them). The loss is the mean squared error of the
 * standardised displacement over the d real outputs; the update is Adam
 * (Kingma & Ba 2015) with a cosine learning-rate decay.
 * All pointers of these calls are device pointers unless stated.
 * ------------------------------------------------------------------------- */
typedef struct smap_proposal smap_proposal;

/* Creates a proposal for a model (parameters as in smap_config, host memory),
 * weights uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from `seed`. */
smap_status smap_proposal_create(int model, const double* params, int n_params, uint64_t seed, void* stream,
                                 smap_proposal** out);
void smap_proposal_destroy(smap_proposal* p);
smap_status smap_proposal_dims(const smap_proposal* p, int* in, int* out, int* hidden, long* n_params);
/* Host copies of the FP32 parameters / normalisation (either may be NULL). */
smap_status smap_proposal_get_weights(smap_proposal* p, float* theta, float* norm);
smap_status smap_proposal_set_weights(smap_proposal* p, const float* theta, const float* norm);
/* Normalisation from data: feature column means and standard deviations;
 * target column means and standard deviations, each standard deviation
 * floored at 1% of the largest one among the d outputs. */
smap_status smap_proposal_fit_normalization(smap_proposal* p, const float* feat, const float* targ, long rows);
/* disp [rows][d] = displacement predicted for feat [rows][32]. Synchronous. */
smap_status smap_proposal_forward(smap_proposal* p, const float* feat, long rows, float* disp);
/* One forward and backward pass over all `rows` (no update): gradient of the
 * loss w.r.t. the parameters (host [n_params], may be NULL) and the loss
 * (host, may be NULL). */
smap_status smap_proposal_loss_grad(smap_proposal* p, const float* feat, const float* targ, long rows,
                                    float* grad, double* loss);
/* `steps` Adam steps on minibatches of `batch` rows drawn (Philox) from the
 * n_rows training rows; learning rate decays from lr to lr_final; loss_curve
 * (host [steps], may be NULL) receives each minibatch loss. */
smap_status smap_proposal_train(smap_proposal* p, const float* feat, const float* targ, long n_rows, int steps,
                                int batch, double lr, double lr_final, float* loss_curve);
const char* smap_proposal_last_error(const smap_proposal* p);

/* Training rows from the handle's last run (smap_run_batch with no proposal
 * attached): for every sequence b, step t <= T_b and particle i < N_b, the
 * features of the plain initialisation u and the target x_t^i - u. Rows are
 * ordered by (b, t, i). feat [max_rows][32], targ [max_rows][16] (device);
 * *rows receives the number written; SMAP_E_INVAL if max_rows is too small. */
smap_status smap_proposal_capture(smap_proposal* p, smap_handle* h, float* feat, float* targ, long max_rows,
                                  long* rows);

/* Debug / parity: one inference forward like smap_proposal_forward, with
 * `wait_ns` nanoseconds (global timer) as the limit of every bounded wait of
 * the tensor-core kernel instead of the default 2 s. stall = 1 makes the
 * MMA-issuing thread first wait on a barrier that nothing completes, so that
 * wait runs out before any MMA is issued and the kernel's give-up path runs
 * (the other warps' waits then run out too). Returns SMAP_E_TIMEOUT when a
 * wait ran out (disp not written); the proposal stays usable. */
smap_status smap_debug_proposal_forward(smap_proposal* p, const float* feat, long rows, float* disp,
                                        uint64_t wait_ns, int stall);

/* Attaches a proposal to a handle (p = NULL detaches): smap_run_batch then
 * initialises each step from u + MLP(u, z_t) and runs L_learned SVGD
 * iterations, one graph-captured launch sequence per time step. The proposal
 * must outlive the attachment. */
smap_status smap_set_proposal(smap_handle* h, smap_proposal* p, int L_learned);

/* Kernel variant (particles per thread, block-size bound, threads per
 * particle) used by the step kernels. With threads per particle > 1 the lanes
 * of a group split one particle's sums over the other particles (shorter
 * serial chains: the built-in choice when there are fewer sequences than SMs);
 * those variants sum in a different order, so their results agree with the
 * others to rounding, not bit for bit.
 * smap_autotune times every compiled variant on the first min(B, sample)
 * sequences for `steps` steps of y_all (layout as in smap_run_batch, host or
 * device per on_device) and keeps the fastest; the handle is reset afterwards.
 * variant < 0 in smap_set_variant restores the built-in heuristic. */
smap_status smap_autotune(smap_handle* h, const float* y_all, int sample, int steps,
                          int on_device, int* chosen_variant, float* ms_per_variant,
                          int n_ms);
smap_status smap_set_variant(smap_handle* h, int variant);
int smap_num_variants(void);
smap_status smap_variant_info(int variant, int* particles_per_thread, int* max_threads,
                              int* threads_per_particle);
smap_status smap_get_variant(const smap_handle* h, int* variant, int* threads, int* grid);

/* Debug / parity entry points (host pointers, synchronous).
 * smap_debug_svgd: n_iters SVGD iterations at step t of every sequence, from
 * the given initial particles x_init [B][N][d] with the prior built from the
 * previous set x_prev [B][n_prev][d] (n_prev = 1 and t = 1: x_prev holds
 * x_0^true, whose transition is taken in FP64 from the handle's x0 instead),
 * observation y [B][dy], and for the MAP-conditioned prior the previous
 * scores phi_prev [B][n_prev] FP64 (NULL = zeros). Writes x_out [B][N][d] and
 * the bandwidth of each iteration h_out [B][n_iters] (may be NULL). Does not
 * change the handle's state. */
smap_status smap_debug_svgd(smap_handle* h, int t, const float* x_prev, int n_prev,
                            const float* x_init, const float* y, int n_iters,
                            float* x_out, float* h_out, const double* phi_prev);

/* Raw Philox-4x32-10 words for counters (c0 + k, c1, c2, c3), k < n, key
 * (key0, key1): out [n][4]; and the standard normals the step kernels draw
 * for (seed, seq, t, particles i0..i0+n-1, dimension d): normals [n][d]. */
smap_status smap_debug_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                              uint32_t key0, uint32_t key1, int n, uint32_t* out);
smap_status smap_debug_normals(uint64_t seed, uint32_t seq, uint32_t t, uint32_t i0,
                               int n, int d, float* normals);

/* Debug build only (compiled with SMAP_DEBUG, where every shared-memory row
 * access and the global sequence / step / particle indices are checked, a
 * failed check is recorded and the access skipped, and the calls that launch
 * the kernels return SMAP_E_INVAL naming the failed check): one checked row
 * load at `index` from a shared array of `rows` rows (1..1024) filled with
 * 1.0. value receives what the load returned (1.0, or 0.0 when the check
 * failed), code and at the failed check's code (0: none; 1: a row index)
 * and index. Other builds return SMAP_E_UNSUPPORTED. */
smap_status smap_debug_bounds_probe(int rows, int index, float* value, int* code, int* at);

/* The double-float functions the recursion's scores use (about 48-bit
 * results computed on the FP32 pipe): fn 0 exp (|x| < 60), 1 log (x > 0
 * normal), 2 sqrt (x > 0), of n FP64 inputs (each split into an FP32 pair),
 * returned as FP64. Host arrays; synchronous. */
smap_status smap_debug_df(int fn, const double* in, int n, double* out);

/* Device times of the last smap_run_batch, in milliseconds, from CUDA events
 * recorded on the handle's stream inside its graph: seq_kernel_ms around the
 * persistent step kernel alone, batch_ms around the whole device work (state
 * reset, step kernel, backtracking). Either pointer may be NULL. */
smap_status smap_last_kernel_ms(smap_handle* h, float* seq_kernel_ms, float* batch_ms);

/* How the exact median of the bandwidth rule was found since the last reset,
 * batched run or smap_debug_svgd call, summed over SVGD iterations (counts:
 * host [4]): counts[0] by the bracket around the previous median, counts[1]
 * by the log-histogram locate (new step, or a bracket that held too many
 * keys), counts[2] by the radix-select fallback, counts[3] how many of
 * counts[1] needed the second, refining histogram (more than 2048 keys in the
 * located bins). Synchronises the stream. */
smap_status smap_debug_median_stats(smap_handle* h, int* counts);

/* Debug / parity: while xinit_all is set (device [B][max_T][N][d] FP32, owned
 * by the caller and alive while it is set), smap_run_batch with a proposal
 * attached also copies every step's initial particles x^(0) = u + MLP(u, z_t)
 * into row [b][t-1] (rows of steps a sequence does not run hold what the
 * network computed for them). NULL stops the recording. Either change
 * re-records the batched run's graph at its next call. */
smap_status smap_debug_record_learned_init(smap_handle* h, float* xinit_all);

/* Counters of the forward recursion (Eq. forward_recursion) over the step
 * launches since the last call (host [3]; reading resets them): counts[0]
 * particle-steps scored, counts[1] of those whose best predecessor the FP32
 * screen could not prove unique (a near-tie: every candidate within the
 * screen's rounding bound is scored exactly), counts[2] exact candidate
 * scores computed. Synchronises the stream. */
smap_status smap_debug_recursion_stats(smap_handle* h, unsigned long long* counts);

/* Kernel launches the library has issued since load (its own kernels only). */
uint64_t smap_kernel_launches(void);

const char* smap_status_string(smap_status s);
const char* smap_last_error(const smap_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* SMAP_H */
