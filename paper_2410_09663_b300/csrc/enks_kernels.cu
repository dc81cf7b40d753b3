// enks_kernels.cu -- the ensemble Kalman analysis of Kalman-MPC on one GPU.
//
//   means     Eq. (mathcalX-prediction-sample-mean), Eq. (Ybar-sample-mean-cov)
//   cov       Sigma^Y and Sigma^{XY} of Eq. (Ybar-sample-mean-cov) as one
//             split-K GEMM over the N*m (member, column) samples; the common
//             factor lambda/N is dropped because it cancels in K
//   gain      K = Sigma^{XY} (Sigma^Y)^{-1} by Cholesky, Eq.
//             (ensemble-based-Kalman-update-samplewise)
//   update    X^i <- X^i + K (Ybar_t - Y^i), Y^i = H X^i + V^i, Eq. (Ybar-samples)
//
// Every kernel reads member rows through a row-offset table, so one set of
// kernels serves the U-history layout, the full-history layout and
// caller-provided ensembles.
#include <type_traits>

#include "oic_internal.cuh"
#include "tc_tf32.cuh"

namespace oic {
namespace {

// ------------------------------------------------------------------ init
// Four consecutive elements per thread (m % 4 == 0, so rows and members
// start on 16-byte boundaries); the noise of a quad is one Philox block when
// it is drawn in place.
__global__ void init_kernel(float* __restrict__ E, long ms, int n, int m, int l, int x_row0, int u_row0,
                            const float* __restrict__ X_k, const float* __restrict__ U_prev, NoiseSrc W0)
{
    pdl_begin();
    const int i = blockIdx.y;
    float* Ei = E + (long)i * ms;
    for (int e = 4 * (blockIdx.x * blockDim.x + threadIdx.x); e < (n + l) * m; e += 4 * gridDim.x * blockDim.x) {
        if (e < n * m) {
            *reinterpret_cast<float4*>(Ei + (long)x_row0 * m + e) = *reinterpret_cast<const float4*>(X_k + e);
        } else {
            const int r = e - n * m;
            const float4 u = *reinterpret_cast<const float4*>(U_prev + r);
            const float4 w = noise4(W0, (long)i * l * m + r);
            *reinterpret_cast<float4*>(Ei + (long)u_row0 * m + r) =
                make_float4(u.x + w.x, u.y + w.y, u.z + w.z, u.w + w.w);
        }
    }
}

__global__ void u_advance_kernel(float* __restrict__ E, long ms, int m, int l, int u_from, int u_to, NoiseSrc W)
{
    pdl_begin();
    const int i = blockIdx.y;
    float* Ei = E + (long)i * ms;
    for (int e = 4 * (blockIdx.x * blockDim.x + threadIdx.x); e < l * m; e += 4 * gridDim.x * blockDim.x) {
        const float4 u = *reinterpret_cast<const float4*>(Ei + (long)u_from * m + e);
        const float4 w = noise4(W, (long)i * l * m + e);
        *reinterpret_cast<float4*>(Ei + (long)u_to * m + e) = make_float4(u.x + w.x, u.y + w.y, u.z + w.z, u.w + w.w);
    }
}

// ----------------------------------------------------------------- stats
// Anomaly products without a separate means pass.  With l_i the value of a
// left row (active state rows a < R, then the p perturbed-observation rows)
// and y_i that of an observation row, both shifted by member 0's value at
// the same (row, column):
//   S1[a][j] = sum_i (l_i - l_0)[a][j]
//   S2[a][c] = sum_i sum_j (l_i - l_0)[a][j] (y_i - y_0)[c][j]
// and  sum_i sum_j (l_i - lbar)(y_i - ybar)^T = S2 - (1/N) sum_j S1[a][j] S1y[c][j]
// exactly.  The shifted values are of the ensemble-spread scale, so the FP32
// accumulation never subtracts two large means (the correction term is of
// the same size as S2).  Split-K over members; CTAs of the first row tile
// also write the innovations D^i = Ybar - Y^i (prior values) for the update.
constexpr int SBM = 64, SBN = 72, SPAD = 4;
constexpr int S_TX = 18, S_TY = 16, S_NT = S_TX * S_TY;   // 4 rows x 4 columns per thread

__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

// Output tile SBM x SBN: thread (ty, tx) owns rows 4 ty .. 4 ty + 3 and the
// columns tx + S_TX v (v < 4).  Strided columns keep the 16-byte shared reads
// of B conflict-free (8 consecutive lanes read 8 consecutive rows; the row
// stride m + 4 places them in distinct 16-byte bank groups).  Tiles are
// stored k-contiguous ([row][m + 4]); member 0's values (the shift) sit in
// shared memory next to them.  QA / QB: 16-byte loader chunks per thread.
template <int QA, int QB>
__global__ void __launch_bounds__(S_NT)
stats_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V,
             const float* __restrict__ Yx, const float* __restrict__ Yu, int n_yx, float* __restrict__ part1,
             float* __restrict__ part2, float* __restrict__ Dbuf, int splits)
{
    pdl_begin();
    constexpr int NT = S_NT;
    extern __shared__ __align__(16) float sm[];
    const int R = act.count, p = obs.count, M = R + p;
    const int ld = m + SPAD;
    float* As = sm;                               // [SBM][ld]  (k contiguous)
    float* Bs = As + SBM * ld;                    // [SBN][ld]
    float* A0 = Bs + SBN * ld;                    // member 0, same layout
    float* B0 = A0 + SBM * ld;
    const int bm0 = blockIdx.x * SBM, bn0 = blockIdx.y * SBN, sidx = blockIdx.z;
    const int i0 = (int)((long)sidx * N / splits), i1 = (int)((long)(sidx + 1) * N / splits);
    const int tid = threadIdx.x, tx = tid % S_TX, ty = tid / S_TX;
    const int m4 = m / 4;
    const bool do_s1 = blockIdx.y == 0, do_d = blockIdx.x == 0 && Dbuf != nullptr;

    // loader chunks: consecutive threads take consecutive 16-byte pieces of a
    // row.  Row offsets and the noise source are resolved once: off < 0 marks
    // an empty chunk, vsel 0 no noise, 1 Va, 2 Vb.
    long aoff[QA], boff[QB];
    int aj[QA], bj[QB], avs[QA], bvs[QB], ar[QA], br[QB];
    long avo[QA], bvo[QB];
    float4 pa[QA], pb[QB], s1[QA];
    const float4 Z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int pb_rows = p - obs.nc - V.pa;              // V rows of Vb per member
    auto resolve = [&](int a, long& off, int& vs, long& vo) {
        vs = 0; vo = 0;
        if (a < R) { off = (long)act.rows[a] * m; return; }
        const int c = a - R;
        off = (long)obs.rows[c] * m;
        if (!V.a.live() || c >= p - obs.nc) return;   // constraint rows carry their noise in E
        if (c < V.pa) { vs = 1; vo = (long)c * m; }
        else { vs = 2; vo = (long)(c - V.pa) * m; }
    };
#pragma unroll
    for (int q = 0; q < QA; ++q) {
        const int e = tid + NT * q;
        ar[q] = e < SBM * m4 ? e / m4 : -1;
        aj[q] = 4 * (e % m4);
        const int a = bm0 + ar[q];
        aoff[q] = -1;
        avs[q] = 0; avo[q] = 0;
        if (ar[q] >= 0 && a < M) resolve(a, aoff[q], avs[q], avo[q]);
        s1[q] = Z;
    }
#pragma unroll
    for (int q = 0; q < QB; ++q) {
        const int e = tid + NT * q;
        br[q] = e < SBN * m4 ? e / m4 : -1;
        bj[q] = 4 * (e % m4);
        const int c = bn0 + br[q];
        boff[q] = -1;
        bvs[q] = 0; bvo[q] = 0;
        if (br[q] >= 0 && c < p) resolve(R + c, boff[q], bvs[q], bvo[q]);
    }
    auto value = [&](int i, long off, int vs, long vo, int j) {
        float4 x = *reinterpret_cast<const float4*>(E + (long)i * ms + off + j);
        if (vs == 1) x = f4add(x, noise4(V.a, (long)i * V.pa * m + vo + j));
        else if (vs == 2) x = f4add(x, noise4(V.b, (long)i * pb_rows * m + vo + j));
        return x;
    };
    // member 0 (the shift) into shared memory
#pragma unroll
    for (int q = 0; q < QA; ++q)
        if (ar[q] >= 0) *reinterpret_cast<float4*>(A0 + ar[q] * ld + aj[q]) = aoff[q] >= 0 ? value(0, aoff[q], avs[q], avo[q], aj[q]) : Z;
#pragma unroll
    for (int q = 0; q < QB; ++q)
        if (br[q] >= 0) *reinterpret_cast<float4*>(B0 + br[q] * ld + bj[q]) = boff[q] >= 0 ? value(0, boff[q], bvs[q], bvo[q], bj[q]) : Z;
    auto fetch = [&](int i) {
#pragma unroll
        for (int q = 0; q < QA; ++q) pa[q] = aoff[q] >= 0 ? value(i, aoff[q], avs[q], avo[q], aj[q]) : Z;
#pragma unroll
        for (int q = 0; q < QB; ++q) pb[q] = boff[q] >= 0 ? value(i, boff[q], bvs[q], bvo[q], bj[q]) : Z;
    };
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;

    if (i0 < i1) fetch(i0);
    for (int i = i0; i < i1; ++i) {
        // shift by member 0 (each thread reads back only what it wrote)
#pragma unroll
        for (int q = 0; q < QA; ++q)
            if (ar[q] >= 0) {
                const float4 d = f4sub(pa[q], *reinterpret_cast<const float4*>(A0 + ar[q] * ld + aj[q]));
                *reinterpret_cast<float4*>(As + ar[q] * ld + aj[q]) = d;
                s1[q] = f4add(s1[q], d);
            }
#pragma unroll
        for (int q = 0; q < QB; ++q)
            if (br[q] >= 0) {
                const float4 d = f4sub(pb[q], *reinterpret_cast<const float4*>(B0 + br[q] * ld + bj[q]));
                *reinterpret_cast<float4*>(Bs + br[q] * ld + bj[q]) = d;
                const int c = bn0 + br[q];
                if (do_d && c < p) {
                    const float4 ref = c >= p - obs.nc ? Z   // constraint rows: reference 0
                                       : *reinterpret_cast<const float4*>(
                                             (c < n_yx ? Yx + (long)c * m : Yu + (long)(c - n_yx) * m) + bj[q]);
                    *reinterpret_cast<float4*>(Dbuf + ((long)i * p + c) * m + bj[q]) = f4sub(ref, pb[q]);
                }
            }
        __syncthreads();
        if (i + 1 < i1) fetch(i + 1);            // next member's loads overlap the products
#pragma unroll 2
        for (int k = 0; k < m; k += 4) {
            float4 av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = *reinterpret_cast<const float4*>(As + (4 * ty + u) * ld + k);
#pragma unroll
            for (int v = 0; v < 4; ++v) bv[v] = *reinterpret_cast<const float4*>(Bs + (tx + S_TX * v) * ld + k);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    acc[u][v] = fmaf(av[u].x, bv[v].x, acc[u][v]);
                    acc[u][v] = fmaf(av[u].y, bv[v].y, acc[u][v]);
                    acc[u][v] = fmaf(av[u].z, bv[v].z, acc[u][v]);
                    acc[u][v] = fmaf(av[u].w, bv[v].w, acc[u][v]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int a = bm0 + 4 * ty + u;
        if (a >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = bn0 + tx + S_TX * v;
            if (c < p) part2[((long)sidx * M + a) * p + c] = acc[u][v];
        }
    }
    if (do_s1) {
#pragma unroll
        for (int q = 0; q < QA; ++q) {
            const int a = bm0 + ar[q];
            if (ar[q] >= 0 && a < M)
                *reinterpret_cast<float4*>(part1 + ((long)sidx * M + a) * m + aj[q]) = s1[q];
        }
    }
}

// Sum over split-K partials, 32 consecutive outputs per CTA: warp w adds the
// splits w, w + 8, ... (coalesced), then the 8 partial sums are combined.
__device__ __forceinline__ float split_sum(const float* __restrict__ part, long stride, int splits, int idx,
                                           bool ok, float (*red)[33])
{
    const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
    float s = 0.f;
    if (ok) {
        // four splits' loads in flight before they are added (same order)
        int k = w;
        for (; k + 24 < splits; k += 32) {
            const float v0 = part[(long)k * stride + idx], v1 = part[(long)(k + 8) * stride + idx];
            const float v2 = part[(long)(k + 16) * stride + idx], v3 = part[(long)(k + 24) * stride + idx];
            s += v0;
            s += v1;
            s += v2;
            s += v3;
        }
        for (; k < splits; k += 8) s += part[(long)k * stride + idx];
    }
    red[w][ln] = s;
    __syncthreads();
    float t = 0.f;
    if (w == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][ln];
    return t;
}

// S1[a][j] = sum over splits of part1; with S1oT also the rows a >= R
// transposed, S1oT[j][a - R] (p = M - R columns), for coalesced reads in the
// finalisation.  OT = double for the FP64 finalisation (converted once here,
// not once per use on the FP64 pipe).
template <typename OT>
__global__ void __launch_bounds__(256) s1_reduce_kernel(const float* __restrict__ part1, int splits, int M, int m,
                                                        OT* __restrict__ S1, OT* __restrict__ S1oT, int R)
{
    pdl_begin();
    __shared__ float red[8][33];
    const int idx = blockIdx.x * 32 + threadIdx.x % 32;
    const bool ok = idx < M * m;
    const float t = split_sum(part1, (long)M * m, splits, idx, ok, red);
    if (threadIdx.x < 32 && ok) {
        S1[idx] = (OT)t;
        const int a = idx / m;
        if (S1oT != nullptr && a >= R) S1oT[(long)(idx - a * m) * (M - R) + (a - R)] = (OT)t;
    }
}

// C[a][c] = scale (sum over splits of part2 - (1/N) sum_j S1[a][j] S1[R + c][j])
// (S1 == nullptr: the partials already have the means removed).
// F64: the split sum, the mean correction and the subtraction in FP64 (the
// mixed-precision mode's FP64 anomaly step); else FP32 with an FP64 result.
template <bool F64>
__global__ void __launch_bounds__(256) cov_finalize_kernel(const float* __restrict__ part2,
                                                           const typename std::conditional<F64, double, float>::type* __restrict__ S1,
                                                           const typename std::conditional<F64, double, float>::type* __restrict__ S1o,
                                                           int splits, int M, int p, int m, int N,
                                                           double* __restrict__ C, double scale, int so_c, int so_j,
                                                           float* __restrict__ cyy32, int R, int ld32)
{
    pdl_begin();
    using T = typename std::conditional<F64, double, float>::type;
    __shared__ T red[8][33], cred[8][33];
    const int idx = blockIdx.x * 32 + threadIdx.x % 32;
    const bool ok = idx < M * p;
    const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
    T sp = 0, cp = 0;
    if (ok) {
        // four splits' loads in flight before they are added (same order)
        const long st = (long)M * p;
        int k = w;
        for (; k + 24 < splits; k += 32) {
            const float v0 = part2[k * st + idx], v1 = part2[(k + 8) * st + idx];
            const float v2 = part2[(k + 16) * st + idx], v3 = part2[(k + 24) * st + idx];
            sp += (T)v0;
            sp += (T)v1;
            sp += (T)v2;
            sp += (T)v3;
        }
        for (; k < splits; k += 8) sp += (T)part2[k * st + idx];
        if (S1 != nullptr) {                      // one-pass products: the mean term, columns j = w, w + 8, ...
            const int a = idx / p, c = idx % p;
            const T* x = S1 + (long)a * m;
            const T* y = S1o + (long)c * so_c;         // so_j = 1: row-major; so_c = 1: transposed
            T d0 = 0, d1 = 0;
            int j = w;
            for (; j + 8 < m; j += 16) {
                d0 = fma((T)x[j], (T)y[(long)j * so_j], d0);
                d1 = fma((T)x[j + 8], (T)y[(long)(j + 8) * so_j], d1);
            }
            if (j < m) d0 = fma((T)x[j], (T)y[(long)j * so_j], d0);
            cp = d0 + d1;
        }
    }
    red[w][ln] = sp;
    cred[w][ln] = cp;
    __syncthreads();
    if (threadIdx.x < 32 && ok) {
        T t = 0, corr = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            t += red[q][ln];
            corr += cred[q][ln];
        }
        corr /= (T)N;
        const double v = (double)(t - corr) * scale;
        C[idx] = v;
        // rows R.. (Sigma^Y) also as FP32 rows of ld32, the FP32 gain's
        // shared-memory layout (one bulk copy there)
        if (cyy32 != nullptr && idx >= R * p) cyy32[(idx / p - R) * ld32 + idx % p] = (float)v;
    }
}

// ------------------------------------------------------------------ gain
// K = Cxy Cyy^{-1}, written transposed: Kt = K^T = Cyy^{-1} Cxy^T, [p][R].
//
// Cyy = U^T U (Cholesky, FP32), then per gain row a: U^T z = Cxy[a]^T
// (forward) and U k = z (backward), Kt[.][a] = k.  Each CTA factors Cyy
// itself in shared memory, blocked by panels of 8 rows, one CTA barrier per
// panel.  Panel j's rank-8 update A[i][c] -= sum_d U[j0+d][i] U[j0+d][c]
// goes to panel j+1's rows first (one row per worker warp), which then
// signal the factor warp on a named barrier; the factor warp factors that
// panel (its 8 x 8 diagonal block read into every lane and factored there
// redundantly, so the pivot chain has no shuffles in it; each lane then forms
// the panel's U rows for its own columns; a pivot <= 0 means "not positive
// definite") while the workers update the remaining rows (two at a time,
// their loads in flight together) and run their forward substitutions.
// Workers 0-2 (warps 1-3, one per sub-partition) solve gain rows
// a = 3 b + w: lane t holds elements t + 32 s (s < SL); the forward
// substitution takes one block of eight per panel inside the loop, the
// backward one follows, eight elements per block from the bottom.  Only U's
// upper rows are stored: U[i][c] with lane = i (ld odd) reads conflict-free
// for the backward updates.  Three rows per CTA rather than nine: the
// backward substitutions, which issue-bound the kernel's tail, then run one
// warp per scheduler (the factorisation is repeated in 3x as many CTAs,
// which the GPU has to spare).
//
// Warp roles: warp 0 factors; warps 4 and 8, which share its scheduler
// (warp w issues from sub-partition w mod 4), stay idle; the other nine are
// the workers.
template <int N>
__device__ __forceinline__ float gsel(const float (&v)[N], int q)
{
    float r = v[0];
#pragma unroll
    for (int i = 1; i < N; ++i) r = q == i ? v[i] : r;
    return r;
}

constexpr int GC_NW = 12;                         // warps per CTA
constexpr int GC_T = 32 * GC_NW;
constexpr int GC_W = 9;                           // worker warps (the trailing updates)
constexpr int GC_R = 3;                           // gain rows per CTA: workers 0-2, one per sub-partition
constexpr int GC_B = 8;                           // panel height = substitution block
constexpr int GC_BAR_PANEL = 1;                   // named barrier: next panel's rows updated
constexpr int GC_TILE = 128 * 128;                // one operand part of the update's gain tile, bytes
constexpr long long GC_WAIT = 4000000000LL;       // bounded wait for the staging copy (~2 s)

__device__ __forceinline__ int gc_worker(int w) { return w & 3 ? w - 1 - (w >> 2) : -1; }

// v = pick ? a : v, kept a select: written as a ternary over an unrolled
// loop, the compiler turns the chain below into an indexed local-memory array
__device__ __forceinline__ void sel_f32(float& v, float a, bool pick)
{
    asm("{ .reg .pred q; setp.ne.s32 q, %2, 0; selp.f32 %0, %1, %0, q; }" : "+f"(v) : "f"(a), "r"((int)pick));
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 8-element block of a substitution: the lanes l0 .. l0+7 of slot `slot`
// hold the block's right-hand sides; every lane receives them.
template <int SL>
__device__ __forceinline__ void block_gather(const float (&b)[SL], int slot, int l0, float (&z)[GC_B])
{
    const float bs = gsel<SL>(b, slot);
#pragma unroll
    for (int d = 0; d < GC_B; ++d) z[d] = __shfl_sync(0xffffffffu, bs, l0 + d);
}
template <int SL>
__device__ __forceinline__ void block_put(float (&b)[SL], int slot, int l0, int lane, const float (&z)[GC_B])
{
    float v = z[0];
#pragma unroll
    for (int d = 1; d < GC_B; ++d) sel_f32(v, z[d], lane - l0 == d);
#pragma unroll
    for (int s = 0; s < SL; ++s)
        if (s == slot && lane >= l0 && lane < l0 + GC_B) b[s] = v;
}

// Factor the panel of rows n0 .. n0+7 (up to date in A) and store its U rows
// and 1 / U[j][j].  Returns true on a pivot <= 0 among the real rows
// (j < p); padding rows become zero.
template <int SL>
__device__ __forceinline__ bool factor_panel(int n0, int p, int pp, int ld, int lane, float* __restrict__ A,
                                             float* __restrict__ rinv)
{
    float P[GC_B][SL], g[GC_B][GC_B];             // the panel (lane = column); its diagonal block
#pragma unroll
    for (int d = 0; d < GC_B; ++d) {
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const int c = lane + 32 * s;
            P[d][s] = c < pp ? A[(n0 + d) * ld + c] : 0.f;
        }
#pragma unroll
        for (int e = d; e < GC_B; ++e) g[d][e] = A[(n0 + d) * ld + n0 + e];
    }
    float rs[GC_B];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < GC_B; ++d) {
        const float piv = g[d][d];
        const bool real = n0 + d < p;
        if (real && !(piv > 0.f)) bad = true;
        rs[d] = real && piv > 0.f ? rsqrt_ftz(piv) : 0.f;
#pragma unroll
        for (int e = d + 1; e < GC_B; ++e) g[d][e] *= rs[d];
#pragma unroll
        for (int e = d + 1; e < GC_B; ++e)
#pragma unroll
            for (int f = e; f < GC_B; ++f) g[e][f] = fmaf(-g[d][e], g[d][f], g[e][f]);
    }
    // U rows of the panel for this lane's columns: row d = (P[d] - sum_{e<d} U[e][d] U[e]) / U[d][d]
#pragma unroll
    for (int d = 0; d < GC_B; ++d)
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            P[d][s] *= rs[d];
#pragma unroll
            for (int e = d + 1; e < GC_B; ++e) P[e][s] = fmaf(-g[d][e], P[d][s], P[e][s]);
        }
#pragma unroll
    for (int d = 0; d < GC_B; ++d)
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const int c = lane + 32 * s;
            if (c >= n0 + d && c < pp) A[(n0 + d) * ld + c] = P[d][s];
        }
    if (lane < GC_B) rinv[n0 + lane] = gsel<GC_B>(rs, lane);
    return bad;
}

// A[i][c] -= sum_d U[j0+d][i] U[j0+d][c] for the columns c >= i of row i
// (U's panel rows in pu, lane = column)
template <int SL>
__device__ __forceinline__ void panel_update_row(float* __restrict__ A, int ld, int p, int j0, int i, int lane,
                                                 const float (&pu)[GC_B][SL])
{
    float q[GC_B];
#pragma unroll
    for (int d = 0; d < GC_B; ++d) q[d] = A[(j0 + d) * ld + i];
    float* ai = A + i * ld;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int c = lane + 32 * s;
        if (c >= i && c < p) {
            float y = 0.f, z = 0.f;
#pragma unroll
            for (int d = 0; d < GC_B; d += 2) {
                y = fmaf(q[d], pu[d][s], y);
                z = fmaf(q[d + 1], pu[d + 1][s], z);
            }
            ai[c] -= y + z;
        }
    }
}

// The same for rows i and i2 (i2 >= p: none) at once, their loads in flight
// together.
template <int SL>
__device__ __forceinline__ void panel_update_rows2(float* __restrict__ A, int ld, int p, int j0, int i, int i2,
                                                   int lane, const float (&pu)[GC_B][SL])
{
    if (i2 >= p) {
        panel_update_row<SL>(A, ld, p, j0, i, lane, pu);
        return;
    }
    float q[GC_B], q2[GC_B];
#pragma unroll
    for (int d = 0; d < GC_B; ++d) {
        q[d] = A[(j0 + d) * ld + i];
        q2[d] = A[(j0 + d) * ld + i2];
    }
    float* ai = A + i * ld;
    float* ai2 = A + i2 * ld;
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int c = lane + 32 * s;
        if (c >= i && c < p) {
            float y = 0.f, z = 0.f;
#pragma unroll
            for (int d = 0; d < GC_B; d += 2) {
                y = fmaf(q[d], pu[d][s], y);
                z = fmaf(q[d + 1], pu[d + 1][s], z);
            }
            ai[c] -= y + z;
        }
        if (c >= i2 && c < p) {
            float y = 0.f, z = 0.f;
#pragma unroll
            for (int d = 0; d < GC_B; d += 2) {
                y = fmaf(q2[d], pu[d][s], y);
                z = fmaf(q2[d + 1], pu[d + 1][s], z);
            }
            ai2[c] -= y + z;
        }
    }
}

template <int SL>
__global__ void __launch_bounds__(GC_T, 1)
gain_chol_kernel(const double* __restrict__ C, int R, int p, float* __restrict__ Kt, int* __restrict__ status,
                 float* __restrict__ Aop, const float* __restrict__ cyy32)
{
    pdl_begin();
    extern __shared__ __align__(16) float gsm[];
    __shared__ __align__(8) uint64_t cmb;          // the bulk copy of Cyy (with cyy32)
    const int pp = (p + GC_B - 1) & ~(GC_B - 1);  // whole panels (zero rows, rinv 0)
    const int ld = pp | 1;
    const int nb = pp / GC_B;
    float* A = gsm;                               // [pp][ld]: Cyy, then U (upper rows)
    float* rinv = A + pp * ld;                    // [pp]: 1 / U[j][j]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const bool factor = w == 0;
    const int wk = gc_worker(w);                  // worker index, -1: not a worker
    const double* Cyy = C + (long)R * p;
    // staging.  With cyy32 (Cyy already in FP32 rows of ld, written by the
    // finalisation) one bulk copy brings the whole [pp][ld] block; otherwise
    // zero the padding, then the worker's gain row and Cyy (each warp rows w,
    // w + 12, ..., the lanes their columns) in rounds of two rows per warp
    // (measured faster than one round of every row)
    const uint32_t cbytes = (uint32_t)(sizeof(float) * pp * ld);   // a multiple of 32 (pp of 8)
    if (cyy32 != nullptr) {
        if (tid == 0) {
            tc::mbar_init(&cmb, 1);
            tc::fence_mbar_init();
            tf32::st_expect_tx(&cmb, cbytes);
            tf32::st_bulk(tc::smem_u32(A), cyy32, cbytes, &cmb);
        }
    } else if (pp > p) {
        for (int e = tid; e < pp * ld; e += GC_T) {
            const int i = e / ld, c = e % ld;
            if (i >= p || c >= p) A[e] = 0.f;
        }
    }
    const int a = blockIdx.x * GC_R + wk;
    const bool mine = wk >= 0 && wk < GC_R && a < R;
    float b[SL];
    {
        constexpr int RW = 2;                                       // rows per warp and round
        double g[SL];
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const int i = lane + 32 * s;
            g[s] = mine && i < p ? __ldg(C + (long)a * p + i) : 0.0;
        }
        for (int i0 = w; cyy32 == nullptr && i0 < p; i0 += GC_NW * RW) {
            double v[RW * SL];
#pragma unroll
            for (int u = 0; u < RW * SL; ++u) {
                const int i = i0 + GC_NW * (u / SL), c = lane + 32 * (u % SL);
                v[u] = i < p && c < p ? __ldg(Cyy + (long)i * p + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < RW * SL; ++u) {
                const int i = i0 + GC_NW * (u / SL), c = lane + 32 * (u % SL);
                if (i < p && c < p) A[i * ld + c] = (float)v[u];
            }
        }
#pragma unroll
        for (int s = 0; s < SL; ++s) b[s] = (float)g[s];
    }
    // the gain rows that read K = 0: the update leaves the ensemble as it is
    auto zero_gain = [&]() {
        if (mine) {
            for (int i = lane; i < p; i += 32) Kt[(long)i * R + a] = 0.f;
            if (Aop != nullptr) {
                char* t0 = reinterpret_cast<char*>(Aop) + (size_t)(a >> 7) * SL * 2 * GC_TILE;
                const int off = tf32::swz(a & 127, lane >> 2) + (lane & 3) * 4;
                for (int s = 0; s < 2 * SL; ++s) *reinterpret_cast<float*>(t0 + (size_t)s * GC_TILE + off) = 0.f;
            }
        }
    };
    __syncthreads();
    if (cyy32 != nullptr) {
        // every thread waits for the copy (bounded); on a timeout thread 0
        // waits once more for the copy in flight before the CTA leaves
        if (__syncthreads_or(!tc::mbar_wait_bounded(&cmb, 0u, GC_WAIT))) {
            if (tid == 0) {
                atomicExch(status, DEV_TIMEOUT);
                tc::mbar_wait_bounded(&cmb, 0u, GC_WAIT);
            }
            zero_gain();
            return;
        }
        if (pp > p) {                             // the padding rows and columns read zero
            for (int e = tid; e < pp * ld; e += GC_T) {
                const int i = e / ld, c = e % ld;
                if (i >= p || c >= p) A[e] = 0.f;
            }
            __syncthreads();
        }
    }
    bool fbad = false;                            // the factor warp: a panel failed
    if (factor) fbad = factor_panel<SL>(0, p, pp, ld, lane, A, rinv);
    // one CTA barrier per panel; it also tells every thread whether a panel failed
    bool failed = __syncthreads_or(fbad);
    for (int j = 0; j < nb; ++j) {
        if (failed) break;
        const int j0 = j * GC_B, n0 = j0 + GC_B;
        const bool next = j + 1 < nb;
        if (factor) {
            if (next) {
                asm volatile("bar.sync %0, %1;" ::"n"(GC_BAR_PANEL), "n"(32 * (GC_W + 1)) : "memory");
                fbad = factor_panel<SL>(n0, p, pp, ld, lane, A, rinv);
            }
        } else if (wk >= 0) {
            float pu[GC_B][SL];                   // panel j's U rows, lane = column
#pragma unroll
            for (int d = 0; d < GC_B; ++d)
#pragma unroll
                for (int s = 0; s < SL; ++s) {
                    const int c = lane + 32 * s;
                    pu[d][s] = c < pp ? A[(j0 + d) * ld + c] : 0.f;
                }
            if (next) {
                // panel j+1's rows first, then tell the factor warp
                if (wk < GC_B && n0 + wk < p) panel_update_row<SL>(A, ld, p, j0, n0 + wk, lane, pu);
                asm volatile("bar.arrive %0, %1;" ::"n"(GC_BAR_PANEL), "n"(32 * (GC_W + 1)) : "memory");
            }
            // the rows from panel j+2 on
            for (int i = n0 + GC_B + wk; i < p; i += 2 * GC_W)
                panel_update_rows2<SL>(A, ld, p, j0, i, i + GC_W, lane, pu);
            // forward substitution, block j of the own gain row: U^T z = b
            if (mine) {
                const int slot = j0 >> 5, l0 = j0 & 31;
                float z[GC_B];
                block_gather<SL>(b, slot, l0, z);
#pragma unroll
                for (int d = 0; d < GC_B; ++d) {
                    const float* ud = A + (j0 + d) * ld;
                    z[d] *= rinv[j0 + d];
#pragma unroll
                    for (int e = d + 1; e < GC_B; ++e) z[e] = fmaf(-ud[j0 + e], z[d], z[e]);
                }
                block_put<SL>(b, slot, l0, lane, z);
#pragma unroll
                for (int s = 0; s < SL; ++s) {
                    const int i = lane + 32 * s;
                    if (i >= n0 && i < pp) {
                        float y = 0.f, x = 0.f;
#pragma unroll
                        for (int d = 0; d < GC_B; d += 2) {
                            y = fmaf(pu[d][s], z[d], y);
                            x = fmaf(pu[d + 1][s], z[d + 1], x);
                        }
                        b[s] -= y + x;
                    }
                }
            }
        }
        failed = __syncthreads_or(fbad);
    }
    if (failed) {                                 // K = 0: the update leaves the ensemble as it is
        if (tid == 0) atomicExch(status, DEV_NOTSPD);
        zero_gain();
        return;
    }
    if (!mine) return;
    // backward: U k = z, blocks of eight from the bottom
    for (int k0 = pp - GC_B; k0 >= 0; k0 -= GC_B) {
        const int slot = k0 >> 5, l0 = k0 & 31;
        float x[GC_B];
        block_gather<SL>(b, slot, l0, x);
#pragma unroll
        for (int dd = 0; dd < GC_B; ++dd) {
            const int d = GC_B - 1 - dd;
            x[d] *= rinv[k0 + d];
#pragma unroll
            for (int e = 0; e < d; ++e) x[e] = fmaf(-A[(k0 + e) * ld + k0 + d], x[d], x[e]);
        }
        block_put<SL>(b, slot, l0, lane, x);
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const int i = lane + 32 * s;
            if (i < k0) {
                const float* ui = A + i * ld + k0;
                float y = 0.f, v = 0.f;
#pragma unroll
                for (int d = 0; d < GC_B; d += 2) {
                    y = fmaf(ui[d], x[d], y);
                    v = fmaf(ui[d + 1], x[d + 1], v);
                }
                b[s] -= y + v;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < SL; ++s) {
        const int i = lane + 32 * s;
        if (i < p) Kt[(long)i * R + a] = b[s];
    }
    if (Aop != nullptr) {
        // the member update's operand: row a of tile a / 128, K chunk s, hi and lo
        // (128-byte-swizzled rows of 32 values; zero beyond p)
        char* t0 = reinterpret_cast<char*>(Aop) + (size_t)(a >> 7) * SL * 2 * GC_TILE;
        const int off = tf32::swz(a & 127, lane >> 2) + (lane & 3) * 4;
#pragma unroll
        for (int s = 0; s < SL; ++s) {
            const float hi = tf32::tf32_rna(b[s]);
            *reinterpret_cast<float*>(t0 + (size_t)s * 2 * GC_TILE + off) = hi;
            *reinterpret_cast<float*>(t0 + ((size_t)s * 2 + 1) * GC_TILE + off) = tf32::tf32_rna(b[s] - hi);
        }
    }
}

size_t gain_chol_smem(int p)
{
    const int pp = (p + GC_B - 1) & ~(GC_B - 1), ld = pp | 1;
    return sizeof(float) * ((size_t)pp * ld + pp);
}

template <int SL>
void gain_chol_launch(const double* C, int R, int p, float* Kt, int* status, cudaStream_t st, float* Aop,
                      const float* cyy32)
{
    const size_t smem = gain_chol_smem(p);
    static DeviceOnce attr_set;
    attr_set.run([] {
        return cudaFuncSetAttribute(gain_chol_kernel<SL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)gain_chol_smem(32 * SL)) == cudaSuccess;
    });
    const int grid = R > 0 ? (R + GC_R - 1) / GC_R : 1;
    pdl_launch(gain_chol_kernel<SL>, grid, GC_T, smem, st, C, R, p, Kt, status, Aop, cyy32);
}

// ---------------------------------------------------------------- update
// E^i[act rows] += K D^i for every member: a GEMM tile of 64 rows x 64
// columns of one member; K is read transposed (Kt[c][a], row length R) and
// D from the buffer the stats pass filled from the prior ensemble.
constexpr int UBM = 64, UBN = 64, UT = 256;

__global__ void __launch_bounds__(UT)
update_kernel(float* __restrict__ E, long ms, int m, RowSet act, const float* __restrict__ Kt, int p,
              const float* __restrict__ Dbuf)
{
    pdl_begin();
    extern __shared__ __align__(16) float sm[];
    const int R = act.count;
    const int ld = UBM + SPAD;
    float* Ks = sm;                               // [p][ld]
    float* Ds = sm + p * ld;                      // [p][ld]
    const int a0 = blockIdx.x * UBM;
    const int ctiles = (m + UBN - 1) / UBN;
    const int i = blockIdx.y / ctiles, j0 = (blockIdx.y % ctiles) * UBN;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int e = tid; e < p * (UBM / 4); e += UT) {
        const int c = e / (UBM / 4), r4 = (e % (UBM / 4)) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        const int a = a0 + r4;
        if ((R & 3) == 0 && a + 3 < R) v = *reinterpret_cast<const float4*>(Kt + (long)c * R + a);
        else {
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            for (int u = 0; u < 4; ++u) if (a + u < R) t[u] = Kt[(long)c * R + a + u];
            v = make_float4(t[0], t[1], t[2], t[3]);
        }
        *reinterpret_cast<float4*>(Ks + c * ld + r4) = v;
    }
    const float* Di = Dbuf + (long)i * p * m;
    for (int e = tid; e < p * (UBN / 4); e += UT) {
        const int c = e / (UBN / 4), j4 = (e % (UBN / 4)) * 4, j = j0 + j4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < m) v = *reinterpret_cast<const float4*>(Di + (long)c * m + j);
        *reinterpret_cast<float4*>(Ds + c * ld + j4) = v;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 4
    for (int c = 0; c < p; ++c) {
        const float4 k4 = *reinterpret_cast<const float4*>(Ks + c * ld + ty * 4);
        const float4 d4 = *reinterpret_cast<const float4*>(Ds + c * ld + tx * 4);
        const float kv[4] = {k4.x, k4.y, k4.z, k4.w}, dv[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(kv[u], dv[v], acc[u][v]);
    }
    const int j = j0 + tx * 4;
    if (j >= m) return;
    float* Ei = E + (long)i * ms;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int a = a0 + ty * 4 + u;
        if (a >= R) continue;
        float4* dst = reinterpret_cast<float4*>(Ei + (long)act.rows[a] * m + j);
        float4 e4 = *dst;
        e4.x += acc[u][0]; e4.y += acc[u][1]; e4.z += acc[u][2]; e4.w += acc[u][3];
        *dst = e4;
    }
}

__global__ void __launch_bounds__(256) block_means_kernel(const float* __restrict__ E, long ms, int N, int m,
                                                          int row0, int rows_per_block, int n_blocks,
                                                          float* __restrict__ out, unsigned long long* tick,
                                                          float* __restrict__ c0, float* __restrict__ c1)
{
    // 32 outputs per CTA (lane = output, coalesced); the members are split
    // over the 8 warps (eight loads in flight each), then summed in shared memory
    pdl_begin();
    if (tick && blockIdx.x == 0 && threadIdx.x == 0) *tick += 1ull;   // after every draw of the solve
    __shared__ float red[8][33];
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    const int idx = blockIdx.x * 32 + ln;
    const bool ok = idx < n_blocks * rows_per_block * m;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (ok) {
        const long off = (long)row0 * m + idx;  // blocks are contiguous rows
        int i = w;
        for (; i + 56 < N; i += 64) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = E[(long)(i + 8 * q) * ms + off];
            s0 += v[0];
            s1 += v[1];
            s2 += v[2];
            s3 += v[3];
            s0 += v[4];
            s1 += v[5];
            s2 += v[6];
            s3 += v[7];
        }
        for (; i < N; i += 8) s0 += E[(long)i * ms + off];
    }
    red[w][ln] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    if (w == 0 && ok) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][ln];
        const float v = t / (float)N;
        out[idx] = v;
        if (idx < rows_per_block * m) {             // block 0 also to the copies
            if (c0) c0[idx] = v;
            if (c1) c1[idx] = v;
        }
    }
}

// d0 = d1 = src (count floats; d1 may be null)
__global__ void __launch_bounds__(256) copy2_kernel(const float* __restrict__ src, float* __restrict__ d0,
                                                    float* __restrict__ d1, int count)
{
    pdl_begin();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const float v = src[i];
        d0[i] = v;
        if (d1) d1[i] = v;
    }
}

}  // namespace

void launch_ensemble_init(float* E, long ms, int N, int n, int m, int l, int x_row0, int u_row0, const float* X_k, const float* U_prev,
                          NoiseSrc W0, cudaStream_t st)
{
    dim3 grid(((n + l) * m / 4 + 255) / 256, N);
    pdl_launch(init_kernel, grid, 256, 0, st, E, ms, n, m, l, x_row0, u_row0, X_k, U_prev, W0);
}

void launch_u_advance(float* E, long ms, int N, int m, int l, int u_from, int u_to, NoiseSrc W, cudaStream_t st)
{
    dim3 grid((l * m / 4 + 255) / 256, N);
    pdl_launch(u_advance_kernel, grid, 256, 0, st, E, ms, m, l, u_from, u_to, W);
}

int stats_splits(int R, int p, int N)
{
    const int tiles = ((R + p + SBM - 1) / SBM) * ((p + SBN - 1) / SBN);
    int s = 148 / tiles;                          // one wave: at most one CTA per SM
    if (s > N) s = N;
    if (s < 1) s = 1;
    return s;
}

size_t stats_smem_bytes(int m) { return sizeof(float) * 2 * (size_t)(SBM + SBN) * (m + SPAD); }

void launch_stats(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
                  const float* Yu, int n_yx, float* part1, float* part2, float* Dbuf, int splits, cudaStream_t st)
{
    const int M = act.count + obs.count, p = obs.count;
    dim3 grid((M + SBM - 1) / SBM, (p + SBN - 1) / SBN, splits);
    const size_t smem = stats_smem_bytes(m);
    static DeviceOnce attr_set;
    attr_set.run([] {
        return cudaFuncSetAttribute(stats_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                   cudaSuccess &&
               cudaFuncSetAttribute(stats_kernel<8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                   cudaSuccess;
    });
    // loader chunks: SBM m / 4 and SBN m / 4 pieces over S_NT threads
    if (m <= 64)
        pdl_launch(stats_kernel<4, 4>, grid, S_NT, smem, st, E, ms, N, m, act, obs, V, Yx, Yu, n_yx, part1, part2, Dbuf,
                                                     splits);
    else
        pdl_launch(stats_kernel<8, 8>, grid, S_NT, smem, st, E, ms, N, m, act, obs, V, Yx, Yu, n_yx, part1, part2, Dbuf,
                                                     splits);
}

// The two reductions after the covariance products are launched without
// programmatic serialisation: with it, their many small CTAs are placed on
// the SMs around the products' persistent grid while it still runs, and the
// 64 x 64 step measured slower (528 against 532 control steps/s device-timed,
// 530 against 545 end to end, on one box).
void launch_s1_reduce(const float* part1, int splits, int M, int m, void* S1, cudaStream_t st, void* S1oT, int R,
                      bool f64)
{
    if (f64)
        plain_launch(s1_reduce_kernel<double>, (M * m + 31) / 32, 256, 0, st, part1, splits, M, m,
                     static_cast<double*>(S1), static_cast<double*>(S1oT), R);
    else
        plain_launch(s1_reduce_kernel<float>, (M * m + 31) / 32, 256, 0, st, part1, splits, M, m,
                     static_cast<float*>(S1), static_cast<float*>(S1oT), R);
}

void launch_cov_finalize_rows(const float* part2, const void* S1_left, const void* S1_obs, int splits, int M, int p,
                              int m, int N, double* C, cudaStream_t st, bool f64, double scale, bool obs_t,
                              float* cyy32, int R)
{
    const int so_c = obs_t ? 1 : m, so_j = obs_t ? p : 1;
    const int total = M * p;
    const int ld32 = gain_chol_ld(p);
    if (f64)
        plain_launch(cov_finalize_kernel<true>, (total + 31) / 32, 256, 0, st, part2,
                     static_cast<const double*>(S1_left), static_cast<const double*>(S1_obs), splits, M, p, m, N, C,
                     scale, so_c, so_j, cyy32, R, ld32);
    else
        plain_launch(cov_finalize_kernel<false>, (total + 31) / 32, 256, 0, st, part2,
                     static_cast<const float*>(S1_left), static_cast<const float*>(S1_obs), splits, M, p, m, N, C,
                     scale, so_c, so_j, cyy32, R, ld32);
}

void launch_cov_finalize(const float* part2, const void* S1, int splits, int R, int p, int m, int N, double* C,
                         cudaStream_t st, bool f64, double scale, const void* S1oT, float* cyy32)
{
    if (S1 != nullptr && S1oT != nullptr) {
        launch_cov_finalize_rows(part2, S1, S1oT, splits, R + p, p, m, N, C, st, f64, scale, true, cyy32, R);
        return;
    }
    const void* S1o = S1 == nullptr ? nullptr
                      : f64 ? static_cast<const void*>(static_cast<const double*>(S1) + (size_t)R * m)
                            : static_cast<const void*>(static_cast<const float*>(S1) + (size_t)R * m);
    launch_cov_finalize_rows(part2, S1, S1o, splits, R + p, p, m, N, C, st, f64, scale, false, cyy32, R);
}


void launch_gain(const double* C, int R, int p, float* K, int* status, cudaStream_t st, float* Aop,
                 const float* cyy32)
{
    switch ((p + 31) / 32) {
    case 1: gain_chol_launch<1>(C, R, p, K, status, st, Aop, cyy32); break;
    case 2: gain_chol_launch<2>(C, R, p, K, status, st, Aop, cyy32); break;
    case 3: gain_chol_launch<3>(C, R, p, K, status, st, Aop, cyy32); break;
    case 4: gain_chol_launch<4>(C, R, p, K, status, st, Aop, cyy32); break;
    default: gain_chol_launch<5>(C, R, p, K, status, st, Aop, cyy32); break;
    }
}

int gain_chol_ld(int p) { return ((p + GC_B - 1) & ~(GC_B - 1)) | 1; }
size_t gain_cyy32_bytes(int p)
{
    const int pp = (p + GC_B - 1) & ~(GC_B - 1);
    return sizeof(float) * (size_t)pp * (pp | 1);
}

void launch_update(float* E, long ms, int N, int m, RowSet act, const float* Kt, int p, const float* Dbuf,
                   cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * (size_t)p * (UBM + SPAD);
    static DeviceOnce attr_set;
    attr_set.run([] {
        return cudaFuncSetAttribute(update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
               cudaSuccess;
    });
    dim3 grid((act.count + UBM - 1) / UBM, N * ((m + UBN - 1) / UBN));
    pdl_launch(update_kernel, grid, UT, smem, st, E, ms, m, act, Kt, p, Dbuf);
}

void launch_block_means(const float* E, long ms, int N, int m, int row0, int rows_per_block,
                        int n_blocks, float* out, cudaStream_t st, unsigned long long* tick, float* c0, float* c1)
{
    const int total = n_blocks * rows_per_block * m;
    pdl_launch(block_means_kernel, (total + 31) / 32, 256, 0, st, E, ms, N, m, row0, rows_per_block, n_blocks, out,
               tick, c0, c1);
}

void launch_copy2(const float* src, float* d0, float* d1, int count, cudaStream_t st)
{
    const int blocks = (count + 1023) / 1024;
    pdl_launch(copy2_kernel, blocks < 1 ? 1 : blocks, 256, 0, st, src, d0, d1, count);
}

}  // namespace oic
