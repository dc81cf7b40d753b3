// oic_internal.cuh -- declarations shared by the library's CUDA sources.
//
// Ensemble layout in the workspace (member-major, one contiguous block per
// member, row-major rows of m floats):
//   U-history mode  rows = [X slot 0 (n) | X slot 1 (n) | U_0 .. U_H (l each)]
//   full history    rows = [X_0 .. X_H (n each)        | U_0 .. U_H (l each)]
// Only these rows are ever touched by an update: the dU rows of the
// augmented state [X; U; dU] (Eq. (virtual-system-compact)) feed neither the
// prediction nor the pseudo-observation, and every row's update depends only
// on its own anomalies (Eq. (ensemble-based-Kalman-update-samplewise)), so
// dropping them leaves every kept row's arithmetic unchanged.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>

#include "oic.h"
#include "philox.cuh"

namespace oic {

// Values of the device status word.
enum : int { DEV_OK = 0, DEV_NOTSPD = 1, DEV_TIMEOUT = 2 };

// cudaFuncSetAttribute acts on the context of the current device only, so a
// kernel's raised shared-memory limit must be set once per device.  Each call
// site keeps one DeviceOnce; run(f) calls f (returning true on success) the
// first time it is reached with each device current, from any host thread.
class DeviceOnce {
  public:
    template <class F>
    bool run(F&& f)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return f();
        std::lock_guard<std::mutex> lock(mu_);
        if (!done_[dev]) done_[dev] = f();
        return done_[dev];
    }

  private:
    static constexpr int kMaxDevices = 64;
    std::mutex mu_;
    bool done_[kMaxDevices] = {};
};

// Programmatic dependent launch: every kernel is launched with programmatic
// stream serialisation, and its first statement lets the next kernel in the
// stream start launching; it then waits until the previous one has finished
// and its writes are visible (pdl_begin: both at once).  The tensor-core
// kernels put their set-up between the two (barrier initialisation, tensor
// memory allocation, copies of the constant weights into shared memory), so
// that it overlaps the previous kernel's last CTAs; nothing before the wait
// reads memory that any kernel writes, or writes memory that any kernel reads.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_begin()
{
    pdl_trigger();
    pdl_wait();
}

// The same launch without programmatic stream serialisation: the kernel
// starts only after the previous one in the stream has completed.
template <typename... K, typename... A>
inline cudaError_t plain_launch(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <typename... K, typename... A>
inline cudaError_t pdl_launch(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Where member i's row r lives: E + i * member_stride + row_off[r] * m.
// For observation rows, the last nc rows are constraint observations: their
// perturbation is already in E and their reference is 0.
struct RowSet {
    const int* rows;   // device: row offsets (in rows) inside a member block
    int count;
    int nc = 0;
};

// Observation perturbation V^i of the p - nc rows before the constraint rows:
// rows c < pa come from a (member stride pa*m), rows pa <= c < p - nc from
// b (member stride (p-nc-pa)*m), each a buffer or drawn in place (NoiseSrc).
// !a.live() means V = 0.
struct ObsNoise {
    NoiseSrc a, b;
    int pa = 0;
};
inline NoiseSrc noise_buf(const float* p)
{
    NoiseSrc s;
    s.buf = p;
    return s;
}
inline ObsNoise obs_noise_buf(const float* Va, const float* Vb, int pa)
{
    ObsNoise o;
    o.a = noise_buf(Va);
    o.b = noise_buf(Vb);
    o.pa = pa;
    return o;
}

// ---------------------------------------------------------------- CNN
// act0[b] = [X^b ; B U^b]  (two planes of n x m), b < Nb.
void launch_cnn_input(const float* X, long x_ms, const float* U, long u_ms, const float* B,
                      float* act0, int Nb, int n, int m, int l, cudaStream_t st);
// One hidden 3x3 layer with tanh: out[b] = tanh(conv(in[b]) + bias).
void launch_conv_hidden(const float* in, int Cin, float* out, int Cout, int Nb, int n, int m,
                        const float* w, const float* bias, cudaStream_t st);
// Last layer (one output channel) fused with the residual:
// Xout[b] = Xin[b] + rs * (conv(in[b]) + bias).
void launch_conv_out_residual(const float* in, int Cin, const float* Xin, long xin_ms, float* Xout,
                              long xout_ms, int Nb, int n, int m, const float* w,
                              const float* bias, float rs, cudaStream_t st);

// ---------------------------------------------------------------- EnKS
// Algorithm 1's ensemble initialisation: E[i][x_row0 ..] = X_k, E[i][u_row0 ..] = U_prev + W0^i.
void launch_ensemble_init(float* E, long ms, int N, int n, int m, int l, int x_row0, int u_row0,
                          const float* X_k, const float* U_prev, NoiseSrc W0, cudaStream_t st);
// E[i][u_to rows] = E[i][u_from rows] + W^i (l x m per member).
void launch_u_advance(float* E, long ms, int N, int m, int l, int u_from, int u_to,
                      NoiseSrc W, cudaStream_t st);
// Shifted anomaly sums (split-K over members): part1[s][a][j] (first column
// tile only) and part2[s][a][c]; the first row tile also writes the
// innovations Dbuf[i][c][j] = Ybar[c][j] - Y^i[c][j].  Rows a < R are active
// state rows, a >= R the perturbed observations; Ybar rows c < n_yx come from
// Yx, the rest from Yu.  m <= 128.
int stats_splits(int R, int p, int N);
size_t stats_smem_bytes(int m);
void launch_stats(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
                  const float* Yu, int n_yx, float* part1, float* part2, float* Dbuf, int splits, cudaStream_t st);
// f64: S1 (and S1oT) as FP64, for the FP64 finalisation.
void launch_s1_reduce(const float* part1, int splits, int M, int m, void* S1, cudaStream_t st,
                      void* S1oT = nullptr, int R = 0, bool f64 = false);
// C = scale (sum_s part2 - S1 S1_Y^T / N)  ([(R + p) x p], Cxy on top, Cyy below).
// (S1 and S1oT in FP64 when f64).  With cyy32, Cyy is also written as FP32
// rows of gain_chol_ld(p) floats (cyy32 holds gain_cyy32_bytes(p); entries
// beyond p are left as they are).
void launch_cov_finalize(const float* part2, const void* S1, int splits, int R, int p, int m, int N, double* C,
                         cudaStream_t st, bool f64 = false, double scale = 1.0, const void* S1oT = nullptr,
                         float* cyy32 = nullptr);
// The same for M left rows whose split sums part2 [splits][M][p] hold alone:
// C[a][c] = scale (sum_s part2[s][a][c] - S1_left[a] . S1_obs[c] / N); obs_t:
// S1_obs is transposed, [m][p] (coalesced reads; launch_s1_reduce's S1oT);
// cyy32: the FP32 copy of rows R.. as above.
void launch_cov_finalize_rows(const float* part2, const void* S1_left, const void* S1_obs, int splits, int M, int p,
                              int m, int N, double* C, cudaStream_t st, bool f64 = false, double scale = 1.0,
                              bool obs_t = false, float* cyy32 = nullptr, int R = 0);
// The FP32 gain's shared-memory layout of Cyy: rows of gain_chol_ld(p)
// floats, gain_cyy32_bytes(p) in all (p rounded up to whole panels).
int gain_chol_ld(int p);
size_t gain_cyy32_bytes(int p);
// Anomaly products on the tensor cores (TF32 hi / lo split, one pass over
// the ensemble): part1 / part2 as launch_stats writes them, so the same
// s1 reduction and finalisation follow.  Bop: stats_tc_bbytes of scratch.
bool stats_tc_supported(int m, int p);
int stats_tc_splits(int M, int N);
int stats_tc_rtiles(int M);
size_t stats_tc_bbytes(int N, int p, int m);
// The innovations go to Dbuf (plain [i][c][m]) or, when Bd is given, to
// the tensor-core update's operand (launch_update_tc).
void launch_stats_tc(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
                     const float* Yu, int n_yx, float* Bop, float* part1, float* part2, float* Dbuf, float* Bd,
                     int splits, int* err, cudaStream_t st);
// The two halves of launch_stats_tc: the observation tiles (and innovations),
// then the products of M left rows, which are the act rows followed by the
// obs rows, cut at M (M = p with act.count = 0: the observed rows alone, for
// Sigma^Y; M = act.count: the state rows alone, for Sigma^XY).
void launch_yprep_tc(const float* E, long ms, int N, int m, RowSet obs, ObsNoise V, const float* Yx, const float* Yu,
                     int n_yx, float* Bop, float* Dbuf, float* Bd, cudaStream_t st);
void launch_stats_tc_rows(const float* E, long ms, int N, int m, RowSet act, RowSet obs, int M, const float* Bop,
                          float* part1, float* part2, int splits, int* err, cudaStream_t st);

// Member update on the tensor cores: E[act rows] += K D from Kt [p][R] and
// the operand tiles yprep wrote (Bd); Aop: update_tc_abytes of scratch.
bool update_tc_supported(int m, int p);
size_t update_tc_abytes(int Rmax, int p);
size_t update_tc_bbytes(int N, int m, int p);
// Kt is turned into the gain tiles Aop first unless the gain kernel already
// wrote them (prep_gain = false).
void launch_update_tc(float* E, long ms, int N, int m, RowSet act, const float* Kt, int p, float* Aop, int max_ctas,
                      const float* Bd, int* err, cudaStream_t st, bool prep_gain = true);
// Mixed-precision gain: FP64 Cholesky of Cyy on a cluster of 8 CTAs into
// L [p][p] (p <= 160) followed by 1 / L_ii [p], then FP64 triangular solves
// per row of Cxy; bad: device flag (not SPD).
void launch_gain64(const double* C, int R, int p, double* L, int* bad, float* Kt, int* status, cudaStream_t st);
// Its two halves: the factorisation (reads only the Cyy rows R .. R+p-1 of
// C) and the substitutions for the R gain rows.
void launch_chol64(const double* C, int R, int p, double* L, int* bad, int* status, cudaStream_t st);
void launch_solve64(const double* C, int R, int p, const double* L, const int* bad, float* Kt, cudaStream_t st);
// Kt = (Cxy Cyy^{-1})^T, [p][R] (FP32 Cholesky, p <= 160); with Aop also the
// member update's TF32 operand tiles of the gain; with cyy32 (the
// finalisation's FP32 copy of Cyy) Cyy is staged by one bulk copy.
void launch_gain(const double* C, int R, int p, float* K, int* status, cudaStream_t st, float* Aop = nullptr,
                 const float* cyy32 = nullptr);
// E^i[act rows] += K D^i for every member.
void launch_update(float* E, long ms, int N, int m, RowSet act, const float* Kt, int p, const float* Dbuf,
                   cudaStream_t st);
// out[b][r][j] = mean_i E[i][row0 + b*rows_per_block + r][j] for blocks b;
// block 0 also to c0 and c1 where given; with tick, *tick += 1 (once).
void launch_block_means(const float* E, long ms, int N, int m, int row0, int rows_per_block,
                        int n_blocks, float* out, cudaStream_t st, unsigned long long* tick = nullptr,
                        float* c0 = nullptr, float* c1 = nullptr);
// d0 = src and, where d1 is given, d1 = src (count floats, one launch).
void launch_copy2(const float* src, float* d0, float* d1, int count, cudaStream_t st);

// Hidden C -> C conv layer on the tensor cores (FP32-accurate fp16 split).
bool conv_tc_supported(int cin, int cout, int m);
size_t conv_tc_packed_bytes(int C);
void conv_tc_pack_weights(const float* w, int C, void* dst_host);
int conv_tc_configure();
void launch_conv_tc(const float* in, float* out, const void* wpk, const float* bias, int C, int Nb, int n,
                    int m, int n_sm, int* err, cudaStream_t st);
// Whole [X; B U] -> 32 -> 32 -> 1 surrogate in one kernel, every layer on the
// tensor cores.  wpk: all three layers' operand tiles (cnn_fused_pack_weights
// from the OIHW weights w1 [32][2][3][3], w2 [32][32][3][3], w3 [1][32][3][3]).
// Returns non-zero if the shape is not supported.
bool cnn_fused_supported(int n_layers, const int* channels, int n, int m, int l);
size_t cnn_fused_packed_bytes();
void cnn_fused_pack_weights(const float* w1, const float* w2, const float* w3, void* dst_host);
// Optional control advance done by the CNN kernels while they read U_{t-1}:
// next[i] = U[i] + w[i] (member stride u_ms for next, l m for w), written
// once per member.  next == nullptr: no advance.
struct UAdvance {
    float* next = nullptr;
    NoiseSrc w;
};
int launch_cnn_fused(const float* X, long x_ms, const float* U, long u_ms, float* Xout, long o_ms,
                     const float* Bmat, int Nb, int n, int m, int l, const float* b1, const float* b2,
                     const float* b3, const void* wpk, float rs, int n_sm, int* err, cudaStream_t st,
                     UAdvance ua = UAdvance());
// Mixed-precision CNN (BF16 operands, FP32 accumulation, FP32 residual):
// one tcgen05 kernel per layer, activations as BF16 rows in the tensor
// core's operand layout.  w[k]: packed tiles of layer k (bf16_pack_layer
// with CI = 16 for k = 0, CO = 16 for the last layer); b[k]: biases padded
// to CO; act_in: first-layer input rows; act[2]: ping-pong activation rows
// (all three zero-initialised: the pad positions are never written).
struct Bf16Net {
    int n_layers = 0, C = 0;
    const void* w[9] = {};
    const float* b[9] = {};
    void* act_in = nullptr;
    void* act[2] = {nullptr, nullptr};
};
bool bf16_supported(int n_layers, const int* channels, int m);
size_t bf16_act_bytes(int N, int n, int m, int C);
size_t bf16_layer_bytes(int CI, int CO);
void bf16_pack_layer(const float* w, int cin, int cout, int CI, int CO, void* dst_host);
int launch_bf16_forward(const Bf16Net& net, const float* X, long x_ms, const float* U, long u_ms, float* Xout,
                        long o_ms, const float* Bmat, int Nb, int n, int m, int l, float rs, int n_sm, int* err,
                        cudaStream_t st);
// Known-answer check of the tcgen05 path: res[0] = mismatches (-1 timeout).
void launch_tc_selftest(int* res, cudaStream_t st);

// Constraint observations of every member at one assimilation time:
// E[i][zrow + r][j] = phi(sum_k G[r][k] S_i[cols[k]][j] - h[r]) + eps[i][r][j]
// with S_i = [X rows from xrow; U rows from urow] of member i (cols[k] < n:
// X row, else U row cols[k] - n), phi(x) = ln(1 + e^{beta x}) / alpha.
// G: [c][nk] packed over the nk columns of [Gx Gu] that are not all zero.
// eps == nullptr: no perturbation.
void launch_constraint_obs(float* E, long ms, int N, int m, int n, int xrow, int urow, int zrow, int c,
                           const float* G, const int* cols, int nk, const float* h, float alpha, float beta,
                           NoiseSrc eps, cudaStream_t st);

// Philox-4x32-10 normal noise (Salmon et al., SC'11) for one solve.
// Philox normals for one solve; the solve index is read from *solve_ctr
// and then incremented on the device (two launches).
void launch_philox_noise(float* out, size_t count_total, unsigned long long seed,
                         unsigned long long* solve_ctr, const size_t* seg_end, const float* seg_sigma,
                         int n_seg, cudaStream_t st, bool tick = true);

}  // namespace oic

#define OIC_CUDA_OK(expr)                                   \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return OIC_ECUDA;           \
    } while (0)
