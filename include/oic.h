/*
 * oic.h -- C ABI of liboic.so: Kalman-MPC (optimal inferential control of a
 * CNN surrogate by a matrix-variate single-pass ensemble Kalman smoother) on
 * one B300 GPU (sm_103a).
 *
 * Method: Vaziri & Fang, "Optimal Inferential Control of Convolutional Neural
 * Networks", arXiv 2410.09663.
 *   CNN surrogate         X_{k+1} = CNN_theta(X_k, U_k), Eq. (1)
 *   virtual system        Eq. (virtual-system), compact form
 *                         Eq. (virtual-system-compact): X̄ = [X; U; dU],
 *                         Ȳ = [X^ref; U^ref], H = [I 0 0; 0 I 0]
 *   ensemble smoother     Eq. (mathcalX-prediction-sample-mean) ..
 *                         Eq. (prediction-mean-cov), Algorithm 1 (Kalman-MPC)
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major float32.  X is n x m (field), U is l x m
 *     (control).  p = n + l observed rows.
 *   - Unless an entry point says "host", array pointers are DEVICE pointers
 *     that must stay valid until the work enqueued on the bound stream has
 *     finished.  Entry points ending in _host take host pointers, copy through
 *     the workspace, and return only after the stream has drained.
 *   - Ownership: weights are copied into the handle at oic_create (the caller
 *     may free its copies afterwards).  The device workspace and the CUDA
 *     stream are owned by the caller (oic_bind); the library never allocates
 *     device memory.
 *   - Errors are returned as oic_status, never thrown and never trapped on
 *     the device.  Device-side failures (a covariance that is not positive
 *     definite) are recorded in a status word inside the workspace; the _host
 *     entry points and oic_sync report it.  On OIC_ENOTSPD the failing update
 *     is skipped (the ensemble keeps its prior) so no NaN propagates.
 *   - Device arrays read as whole rows (noise, and E / V of oic_enks_update)
 *     must be 16-byte aligned; m % 4 == 0 keeps every row aligned after that.
 *   - Calls on one handle must not overlap from several host threads.
 */
#ifndef OIC_H
#define OIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OIC_MAX_LAYERS 8

typedef struct oic_handle oic_handle;

typedef enum {
    OIC_OK = 0,
    OIC_EINVAL = 1,     /* bad size, null pointer, unsupported option        */
    OIC_ENOMEM = 2,     /* workspace too small or host allocation failed     */
    OIC_ECUDA = 3,      /* a CUDA runtime call failed                        */
    OIC_ENOTSPD = 4,    /* Sigma^Y not positive definite in the gain solve   */
    OIC_ETIMEOUT = 5,   /* a bounded device wait gave up                     */
    OIC_ESTATE = 6      /* call order violated (e.g. oic_step before reset)  */
} oic_status;

typedef enum { OIC_PREC_FP32 = 0, OIC_PREC_MIXED = 1 } oic_precision;
typedef enum { OIC_NOISE_HOST = 0, OIC_NOISE_PHILOX = 1 } oic_noise_mode;

/* Problem description (Algorithm 1, Eq. (1), Eq. (virtual-system)). */
typedef struct {
    int n, m;            /* field X is n x m                                  */
    int l;               /* control U is l x m                                */
    int N;               /* ensemble members                                  */
    int H;               /* horizon: updates at t = k+1 .. k+H                */
    int n_layers;        /* conv layers of CNN_theta (1 .. OIC_MAX_LAYERS)    */
    int channels[OIC_MAX_LAYERS + 1]; /* channels[0] = 2 (X and B U),
                                        channels[n_layers] = 1               */
    float residual_scale;             /* X_{k+1} = X_k + s * CNN output        */
    double sigma_w, sigma_vx, sigma_vu; /* noise std of W, V_X, V_U; used by
                                        OIC_NOISE_PHILOX to draw the noise    */
    int precision;       /* oic_precision                                     */
    int keep_full_history; /* 1: keep and update every X block k..k+H (X_hat
                              output available); 0: keep the U blocks and the
                              current X only (same U_hat, less work)          */
    int noise_mode;      /* oic_noise_mode                                    */
    unsigned long long seed; /* OIC_NOISE_PHILOX key                          */
} oic_config;

/* Noise buffer of one solve (OIC_NOISE_HOST), float32, contiguous:
 *   W0 [N][l][m]    initial control spread: U_k^i = U_{k-1} + W0^i, dU_k^i = W0^i
 *   W  [H][N][l][m] process noise of the prediction to t = k+s+1 (row s):
 *                   U_{t} = U_{t-1} + W, dU_t = W   (Eq. (virtual-system))
 *   VX [H][N][n][m] pseudo-observation noise of X at t = k+s+1 (Eq. (Ybar-samples))
 *   VU [H][N][l][m] pseudo-observation noise of U at t = k+s+1
 * Its length in floats is returned by oic_noise_floats. */
size_t oic_noise_floats(const oic_config* cfg);

/* Creates a handle.  conv_w: all layers' weights concatenated, layer k as
 * [channels[k+1]][channels[k]][3][3] (3x3 cross-correlation, zero padding);
 * conv_b: all biases concatenated; B: n x l.  Host pointers, copied.
 * Sizes: n >= 1, 4 <= m <= 128, m % 4 == 0, l >= 1, n + l <= 144, N >= 2,
 * H >= 1, channels in 1 .. 256.  Returns OIC_EINVAL on bad sizes, OIC_ENOMEM on host allocation
 * failure. */
oic_status oic_create(const oic_config* cfg, const float* conv_w, const float* conv_b,
                      const float* B, oic_handle** out);

/* State/input constraints as virtual observations (the paragraph on
 * constraints after Table I of the paper).  A constraint g(X, U) <= 0 is
 * observed as
 *     z_t = phi(g(X̄_t, Ū_t)) + eps_t,   reference 0,
 *     phi(x) = ln(1 + e^{beta x}) / alpha   (softplus barrier, alpha, beta > 0),
 * and z_t joins the pseudo-observation Ȳ_t at every assimilation time
 * t = k+1 .. k+H, so p = n + l + c rows are observed.  The paper's scalar g is
 * evaluated column by column: each of the c constraints is one row of m
 * values, affine in the predicted field and control of the member,
 *     g[r][j] = sum_a Gx[r][a] X_t[a][j] + sum_b Gu[r][b] U_t[b][j] - h[r].
 * (A box |U| <= u on every control entry is c = 2 l rows with Gx = 0,
 * Gu = [I; -I], h = u.)  The rows are observations only: they are not part of
 * the smoothed state.  eps ~ N(0, sigma_z^2): in OIC_NOISE_HOST mode the solve's
 * noise buffer carries VZ [H][N][c][m] after VU (oic_handle_noise_floats), in
 * OIC_NOISE_PHILOX mode it is drawn as a fifth segment after VU, so the other
 * segments are unchanged. */
typedef struct {
    int c;               /* constraint rows, 0 .. 144 - n - l                 */
    const float* Gx;     /* c x n, host, copied at create                     */
    const float* Gu;     /* c x l, host, copied at create                     */
    const float* h;      /* c, host, copied at create                         */
    double alpha, beta;  /* softplus barrier parameters, both > 0             */
    double sigma_z;      /* std of eps (OIC_NOISE_PHILOX)                     */
} oic_constraints;

/* oic_create with constraint rows (cons NULL or cons->c == 0: oic_create).
 * OIC_EINVAL when n + l + c > 144, alpha or beta <= 0, or a pointer is NULL
 * with c > 0. */
oic_status oic_create_constrained(const oic_config* cfg, const float* conv_w, const float* conv_b,
                                  const float* B, const oic_constraints* cons, oic_handle** out);

/* Floats of one solve's OIC_NOISE_HOST noise buffer for this handle:
 * oic_noise_floats(cfg) plus H N c m with constraint rows. */
size_t oic_handle_noise_floats(const oic_handle* h);

/* Device workspace (bytes) the handle needs: ensemble, CNN activations,
 * statistics, gain, plant state and staging for the _host entry points. */
size_t oic_workspace_bytes(const oic_handle* h);

/* Binds caller-owned device memory (>= oic_workspace_bytes, 256-byte
 * aligned) and a CUDA stream (cudaStream_t, NULL = legacy default stream).
 * Copies the weights into the workspace.  May be called again to rebind. */
oic_status oic_bind(oic_handle* h, void* dev_workspace, size_t bytes, void* cuda_stream);

/* Sets the device-resident plant state used by oic_step: X0 (n x m) and the
 * previously applied control U_prev (l x m).  Device pointers. */
oic_status oic_reset(oic_handle* h, const float* X0, const float* U_prev);

/* One receding-horizon solve (Algorithm 1 for one control step) from X_k with the
 * previously applied control U_prev.
 *   X_ref  [(H+1)][n][m] references for times k .. k+H (index 0 unused by the
 *          updates, kept so callers pass a whole window)
 *   U_ref  [l][m]
 *   noise  oic_noise_floats floats (OIC_NOISE_HOST); ignored (may be NULL)
 *          with OIC_NOISE_PHILOX, where the k-th solve draws its noise from
 *          (seed, solve counter)
 *   U_hat  [(H+1)][l][m] out: smoothed control means Û_{k|k:k+H} .. Û_{k+H|k:k+H}
 *   X_hat  [(H+1)][n][m] out, optional (NULL): smoothed field means; requires
 *          keep_full_history (OIC_EINVAL otherwise); block 0 is X_k.
 * Device pointers; asynchronous on the bound stream. */
oic_status oic_solve(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                     const float* U_ref, const float* noise, float* U_hat, float* X_hat);

/* oic_solve with Algorithm 1's optional covariance steps executed (the
 * predicted and the updated state covariance, which the paper lets be skipped
 * because the update does not use them): for s = 1 .. H (t = k + s)
 *   Sigma_pred slot s-1: Sigma^X_{t|t-1} after the prediction to t, whose last
 *                        block row / column are Sigma^{X̄}_{t|t-1} and
 *                        Sigma^{X X̄}_{t|t-1} (Eq. (prediction-cov) ..
 *                        Eq. (prediction-cov-concatenate));
 *   Sigma_post slot s-1: Sigma^X_{t|t} after the update at t
 *                        (Eq. (ensemble-based-Kalman-update-cov));
 * each = (lambda / N) sum_i (X^i - mean)(X^i - mean)^T over the rows the
 * handle keeps at s, pooled over the m columns (lambda = 1 / tr Psi in the
 * paper; Psi is not estimated, so the caller chooses it).  Slot s-1 starts at
 * (s-1) R^2 doubles, R = oic_cov_rows(h, H), and holds the oic_cov_rows(h, s)^2
 * matrix compact, row-major.  Rows kept at s, in order: with keep_full_history
 * the field blocks k+1 .. k+s (n rows each; block k has no spread) then the
 * control blocks k .. k+s (l rows each); otherwise the field at k+s (n rows)
 * then the control blocks k .. k+s.  The dU rows are not kept (the prediction
 * and the observation never read them).
 * scratch: device, 256-byte aligned, >= oic_cov_scratch_bytes(h).  Either
 * Sigma output may be NULL.  Device pointers; asynchronous; FP64 outputs
 * from FP32 products with FP64 split sums and mean correction. */
oic_status oic_solve_cov(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                         const float* U_ref, const float* noise, float* U_hat, float* X_hat, double lambda,
                         double* Sigma_pred, double* Sigma_post, void* scratch, size_t scratch_bytes);
size_t oic_cov_scratch_bytes(const oic_handle* h);
/* Rows kept at s (1 .. H; 0 otherwise). */
int oic_cov_rows(const oic_handle* h, int s);

/* One control step (Algorithm 1: a solve, then U_k applied) on the device-resident plant:
 * solve from the plant state, apply U_k = Û_{k|k:k+H} to the plant
 * X_{k+1} = CNN_theta(X_k, U_k) (the plant is the surrogate itself), and
 * keep U_k as the next step's U_prev.  U_applied [l][m] and X_next [n][m]
 * are optional outputs (NULL to skip).  Device pointers; asynchronous. */
oic_status oic_step(oic_handle* h, const float* X_ref, const float* U_ref, const float* noise,
                    float* U_applied, float* X_next);

/* Host-pointer forms of oic_solve / oic_step / oic_reset: copy inputs in,
 * run, copy outputs out, synchronise the stream, and return the device
 * status (OIC_ENOTSPD if any update of the call failed). */
oic_status oic_solve_host(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                          const float* U_ref, const float* noise, float* U_hat, float* X_hat);
oic_status oic_step_host(oic_handle* h, const float* X_ref, const float* U_ref, const float* noise,
                         float* U_applied, float* X_next);
oic_status oic_reset_host(oic_handle* h, const float* X0, const float* U_prev);

/* X_next[b] = CNN_theta(X[b], U[b]) for b < batch (Eq. (1)); X, X_next
 * [batch][n][m], U [batch][l][m]; batch <= N.  Device pointers; X_next must
 * not overlap X (OIC_EINVAL otherwise).  Uses the workspace's activation
 * buffers, so it must not overlap other calls. */
oic_status oic_cnn_forward(oic_handle* h, int batch, const float* X, const float* U,
                           float* X_next);

/* One ensemble Kalman analysis (Eq. (Ybar-samples) .. Eq.
 * (ensemble-based-Kalman-update)) on a caller-provided ensemble:
 *   E      [N][R][m] in/out, member i's state rows (R <= the handle's
 *          maximum active rows, see oic_max_rows)
 *   obs_rows (host) p_obs row indices of E observed by H (p_obs = n + l)
 *   V      [N][p_obs][m] observation perturbations
 *   Ybar   [p_obs][m] pseudo-observation
 * E^i <- E^i + K (Ybar - (H E^i + V^i)), K = Sigma^{XY} (Sigma^{Y})^{-1}.
 * Device pointers except obs_rows; asynchronous. */
oic_status oic_enks_update(oic_handle* h, int R, const int* obs_rows, float* E, const float* V,
                           const float* Ybar);
int oic_max_rows(const oic_handle* h);

/* Stage profiler: CUDA events recorded on the bound stream around every
 * kernel launch of the selected stages (bit s of stage_mask selects stage s),
 * for up to max_launches launches.  oic_profile_end waits for the stream
 * and writes, per stage, the summed device milliseconds and the launch count
 * (arrays of OIC_NUM_STAGES).  Recording costs no device work beyond the
 * events themselves. */
typedef enum {
    OIC_STAGE_NOISE = 0,       /* Philox noise for one solve                    */
    OIC_STAGE_INIT,            /* Algorithm 1, ensemble initialisation          */
    OIC_STAGE_CNN_INPUT,       /* [X; B U] assembly, Eq. (1)                    */
    OIC_STAGE_CONV_FIRST,      /* first conv layer (2 input channels), tanh     */
    OIC_STAGE_CONV_HIDDEN,     /* hidden -> hidden conv layers, tanh            */
    OIC_STAGE_CONV_OUT,        /* last conv layer + residual                    */
    OIC_STAGE_U_ADVANCE,       /* U_t = U_{t-1} + W                             */
    OIC_STAGE_MEANS,           /* reduction of the anomaly column sums          */
    OIC_STAGE_COV,             /* anomaly products (split-K) and innovations    */
    OIC_STAGE_COV_REDUCE,      /* covariance finalisation                       */
    OIC_STAGE_GAIN,            /* Cholesky + K = Sigma^XY (Sigma^Y)^-1          */
    OIC_STAGE_UPDATE,          /* member-wise update                            */
    OIC_STAGE_BLOCK_MEANS,     /* smoothed output means                         */
    OIC_STAGE_CNN_FUSED,       /* whole CNN step in one kernel (all layers)     */
    OIC_STAGE_CNN_BF16,        /* CNN step in BF16, one kernel per layer        */
    OIC_STAGE_CONSTRAINT,      /* constraint rows z = phi(g(X_t, U_t)) + eps    */
    OIC_STAGE_COV_OUT,         /* optional covariance outputs (oic_solve_cov)   */
    OIC_NUM_STAGES
} oic_stage;
oic_status oic_profile_begin(oic_handle* h, unsigned stage_mask, int max_launches);
oic_status oic_profile_end(oic_handle* h, float* ms, int* launches);

/* Sampling for the profiler started by oic_profile_begin (which resets it to
 * every launch): of the launches of a profiled stage within one solve (and
 * the plant step that follows it in oic_step), counted from 0, only those
 * with index % every == phase are bracketed by events; the others run
 * without event records between them and their neighbours.  A captured step
 * graph is re-captured when the sampling changes.  OIC_EINVAL unless
 * every >= 1 and 0 <= phase < every; OIC_ESTATE when no profile is open. */
oic_status oic_profile_sample(oic_handle* h, int every, int phase);

/* Number of kernels this library has launched in this process. */
unsigned long long oic_launch_count(void);

/* Known-answer check of the tensor-core path on the bound device: a
 * 128 x 64 x 32 fp16 product with FP32 accumulation in tensor memory,
 * compared element by element with CUDA-core results.  result[5] (host):
 * mismatches, then the first mismatch (row, column, got, want).  Returns
 * OIC_OK, OIC_ECUDA on a mismatch, OIC_ETIMEOUT if the product never
 * completed.  Synchronous. */
oic_status oic_selftest(oic_handle* h, int* result);

/* ------------------------------------------------------ scheduling plans
 * How a handle's kernels are laid out on the GPU; the paper has no
 * counterpart (these choices schedule the same arithmetic).  A field of 0
 * means the built-in rule.
 *   stats_splits  member splits of the covariance products of Eq.
 *                 (Ybar-sample-mean-cov): the sums over the N m samples are
 *                 cut into this many partial sums (1 .. limits.stats_splits).
 *                 The partial sums are added in another grouping, so results
 *                 move at the level of FP32 rounding.
 *   update_ctas   CTAs of the persistent tensor-core member update of Eq.
 *                 (ensemble-based-Kalman-update-samplewise), 1 ..
 *                 limits.update_ctas.  Every value gives bit-identical
 *                 results (each output tile is computed the same way).
 *   cnn_ctas      CTAs of the persistent CNN kernels (the fused FP32 kernel,
 *                 the BF16 and the per-layer tensor-core convolutions), 1 ..
 *                 limits.cnn_ctas (the SM count).  Bit-identical results for
 *                 every value. */
typedef struct {
    int stats_splits;
    int update_ctas;
    int cnn_ctas;
} oic_plan;

/* The plan in use with every rule resolved to its value (stats_splits: at
 * the last assimilation time, whose row count is the largest) and, if
 * limits is not NULL, the largest value each field accepts.  OIC_EINVAL on
 * NULL h or plan. */
oic_status oic_get_plan(const oic_handle* h, oic_plan* plan, oic_plan* limits);

/* Sets the plan (0 fields: the rule).  The captured step graphs are dropped
 * and captured again at the next step.  OIC_EINVAL when a field is negative
 * or above its limit. */
oic_status oic_set_plan(oic_handle* h, const oic_plan* plan);

/* Chooses the plan by timing: one field at a time (cnn_ctas, then
 * stats_splits, then update_ctas), each candidate value runs one untimed
 * control step and then `reps` control steps between CUDA events on the
 * bound stream (replays of the step graph in the device-noise mode, launches
 * one by one otherwise), and a value replaces the current one only if it is
 * at least 1% faster.  The inputs of these steps are zero references and
 * device-drawn noise; the plant state, the Philox solve index and the bound
 * stream's ordering are restored afterwards, so the next oic_step continues
 * exactly where the caller left off.  The winner is stored in a process-wide
 * cache keyed by the problem's shape (sizes, channels, precision, history
 * mode, constraint rows, SM count); a later call for the same shape takes it
 * from there without timing unless flags has OIC_TUNE_FORCE.  chosen gets the
 * plan; ms_rule / ms_tuned (may be NULL) the milliseconds per control step
 * with the rule plan and with the chosen plan (both -1 when the plan came from
 * the cache).  Synchronous.  OIC_ESTATE unless h is bound with a plant
 * (oic_reset) and the stage profiler is off; OIC_EINVAL unless 1 <= reps <=
 * 1000. */
#define OIC_TUNE_FORCE 1
oic_status oic_autotune(oic_handle* h, int reps, int flags, oic_plan* chosen, float* ms_rule, float* ms_tuned);

/* Size of the fixed device scratch behind oic_enks_update_static. */
#define OIC_STATIC_SCRATCH_BYTES ((size_t)32 << 20)

/* oic_enks_update for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment variant of the same
 * ensemble Kalman analysis.
 *
 * Who needs it: code that may not call cudaMalloc at all -- a real-time
 * loop that must never reach the allocator after start-up (an allocation can
 * block or fail at any moment), a plug-in whose host application owns all
 * GPU memory and forbids allocations of its own, or an embedding with a
 * fixed memory map.  Such a caller cannot
 * provide the workspace oic_bind needs, so this entry point takes no handle
 * and keeps every intermediate (split-K partials, innovations, covariances,
 * gain, row tables, status) in one device array of OIC_STATIC_SCRATCH_BYTES
 * that the library's CUDA module carries.  Every GPU that loads the library
 * holds that array until the process exits.
 *
 * Arguments (device pointers unless noted; E and V 16-byte aligned):
 *   N, R, m, p   members, state rows, columns, observed rows
 *                (N >= 2, 4 <= m <= 128 with m % 4 == 0, 1 <= p <= 144)
 *   obs_rows     HOST array of p row indices of E (each < R), read during the
 *                call only
 *   E            [N][R][m] in/out: E^i <- E^i + K (Ybar - (E^i[obs_rows] + V^i))
 *   V            [N][p][m] observation perturbations
 *   Ybar         [p][m] pseudo-observation
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream)
 * Returns OIC_OK, OIC_ENOTSPD (the update was skipped; E unchanged),
 * OIC_EINVAL on bad arguments (including E, V or Ybar not in the current
 * device's memory), OIC_ECUDA when the CUDA runtime fails (no device), or
 * OIC_ENOMEM when these sizes need more than
 * OIC_STATIC_SCRATCH_BYTES, which is about
 *   4 (N p m + s (R + p)(m + p) + (R + p) m + p R) + 8 (R + p) p bytes,
 * s = split count (<= 148 / ceil((R + p) / 64)).  It allocates nothing; it
 * copies the row table from host memory and reads the status word back,
 * synchronising the stream before it returns.
 *
 * The first call on each device looks up the scratch's device address with
 * that device current; make that first call before any stream capture.
 * Every call on a device shares the one array and leaves its contents behind
 * (the status word is cleared at the start of each call): calls that overlap
 * on the GPU -- from several host threads or several streams -- race on it
 * and must be serialised by the caller. */
oic_status oic_enks_update_static(int N, int R, int m, int p, const int* obs_rows, float* E,
                                  const float* V, const float* Ybar, void* cuda_stream);

/* Waits for the bound stream and returns (and clears) the device status. */
oic_status oic_sync(oic_handle* h);

/* Milliseconds of device time of the last oic_solve/oic_step (CUDA events
 * around the call on the bound stream; valid after oic_sync). */
float oic_last_ms(oic_handle* h);

/* ------------------------------------------------------- narrow controls
 * The right transformation for controls with fewer columns than the state
 * (the paragraph on narrow controls after the paper's Table I): a control u
 * of mu < m columns enters the method as U = u T, with T (mu x m, T T^T > 0)
 * chosen by the caller (T = [1 ... 1] repeats a column vector), and a
 * smoothed U maps back to u = U T^T (T T^T)^{-1}.  Device pointers,
 * row-major float32, asynchronous on `cuda_stream` except as noted. */

/* U [l][m] = u [l][mu] T [mu][m].  OIC_EINVAL unless 1 <= mu <= m <= 1024
 * and 1 <= l <= 4096. */
oic_status oic_control_expand(const float* u, int l, int mu, const float* T, int m, float* U,
                              void* cuda_stream);

/* u [l][mu] = U [l][m] T^T (T T^T)^{-1}, in FP64 (Cholesky of T T^T, two
 * substitutions per row), rounded to float32 at the end.  Limits 1 <= mu <=
 * 64, mu <= m <= 1024, 1 <= l <= 256.  Synchronises the stream and returns
 * OIC_ENOTSPD (u untouched) if T T^T is not positive definite.  Concurrent
 * calls on several streams share one device status word and must be
 * serialised by the caller. */
oic_status oic_control_reduce(const float* U, int l, int m, const float* T, int mu, float* u,
                              void* cuda_stream);

/* ---------------------------------------------------------------- batching
 * Independent problems stepped together (a deployment extension; the paper
 * solves one problem at a time): one receding-horizon control step of every
 * problem (Algorithm 1) launched as ONE CUDA graph whose branches are the
 * problems' own step graphs, so the GPU runs small problems side by side.
 * Problems may differ in every size; each keeps its own workspace, seed and
 * solve counter, and nothing is shared or reduced across problems, so each
 * result is bit-identical to the same problem stepped alone. */

/* Device addresses of the per-step slots inside h's workspace (valid while
 * h stays bound to the same workspace): inputs X_ref [(H+1)][n][m] and
 * U_ref [l][m], outputs U_applied [l][m] and X_next [n][m] of the last step.
 * Any argument may be NULL.  OIC_ESTATE if h is not bound. */
oic_status oic_io_slots(const oic_handle* h, float** X_ref, float** U_ref, float** U_applied,
                        float** X_next);

/* A problem's state between control steps: the plant X_k [n][m], the last
 * applied control U_{k-1} [l][m] and the Philox solve index -- everything a
 * later oic_step needs besides the handle's configuration.  A server that
 * evicts an idle problem from device memory saves it to the host and loads
 * it into a new handle of the same configuration on re-admission; the next
 * steps are then bit-identical to uninterrupted ones.  Size in bytes: */
size_t oic_state_bytes(const oic_handle* h);
/* Copies the state into host memory `dst` (oic_state_bytes of it) on the
 * bound stream and waits.  OIC_ESTATE if h is not bound or has no plant. */
oic_status oic_save_state(oic_handle* h, void* dst);
/* Sets the state from host memory `src` written by oic_save_state of a
 * handle with the same sizes (asynchronous on the bound stream; src must
 * stay valid until the stream reaches it).  OIC_EINVAL on a size mismatch
 * (the stored sizes are checked), OIC_ESTATE if h is not bound. */
oic_status oic_load_state(oic_handle* h, const void* src);

typedef struct oic_batch oic_batch;

/* Builds the batch graph of `count` handles (1..4096), each bound, with its
 * plant state set (oic_reset) and in OIC_NOISE_PHILOX mode; a handle appears
 * at most once.  The batch launches on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  The batch graph is captured once here: each
 * problem's step on its own branch.  The handles must outlive the batch and
 * stay bound to the same workspaces.  OIC_EINVAL / OIC_ESTATE / OIC_ENOMEM /
 * OIC_ECUDA. */
oic_status oic_batch_create(oic_handle* const* handles, int count, void* cuda_stream, oic_batch** out);

/* One control step of every problem of the batch: each reads its X_ref and
 * U_ref slots and writes its U_applied and X_next slots (oic_io_slots),
 * asynchronously on the batch's stream.  Inputs must be in place, in stream
 * order, before the call. */
oic_status oic_batch_step(oic_batch* b);

/* Chooses one plan for every problem of the batch by timing whole batch
 * steps (the problems share the GPU, so the best choice for a problem alone
 * need not be the best in the mix): CNN CTAs as a fraction of the SMs, the
 * member update's CTAs, and the covariance splits as a fraction of each
 * problem's rule, one field at a time, each candidate a captured batch graph
 * run once untimed and `reps` times between CUDA events on the batch's
 * stream; a value replaces the current one only if at least 1% faster.  The
 * batch graph is captured again with the chosen plans (each handle's plan is
 * set; oic_get_plan reads it).  Every handle's state is restored afterwards;
 * the input slots (oic_io_slots: X_ref, U_ref) hold zeros after the call, so
 * fill them before the next oic_batch_step.  ms_rule / ms_tuned (may be
 * NULL): ms per batch step with the built-in rules and with the chosen
 * plans.  Synchronous.  OIC_EINVAL unless
 * 1 <= reps <= 1000; OIC_ESTATE if a handle's profiler is on. */
oic_status oic_batch_autotune(oic_batch* b, int reps, float* ms_rule, float* ms_tuned);

/* Waits for the batch's stream; returns the first non-OK device status of
 * the handles, in handle order (and clears every handle's status). */
oic_status oic_batch_sync(oic_batch* b);

void oic_batch_destroy(oic_batch* b);

void oic_destroy(oic_handle* h);
const char* oic_status_string(oic_status s);
const char* oic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OIC_H */
