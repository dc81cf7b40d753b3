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
#include "oic_internal.cuh"

namespace oic {
namespace {

__device__ __forceinline__ float obs_noise(const ObsNoise& V, int i, int c, int p, int m, int j)
{
    if (V.Va == nullptr) return 0.f;
    if (c < V.pa) return V.Va[((long)i * V.pa + c) * m + j];
    const int pb = p - V.pa;
    return V.Vb[((long)i * pb + (c - V.pa)) * m + j];
}

__device__ __forceinline__ float4 obs_noise4(const ObsNoise& V, int i, int c, int p, int m, int j)
{
    if (V.Va == nullptr) return make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < V.pa) return *reinterpret_cast<const float4*>(V.Va + ((long)i * V.pa + c) * m + j);
    const int pb = p - V.pa;
    return *reinterpret_cast<const float4*>(V.Vb + ((long)i * pb + (c - V.pa)) * m + j);
}

// ------------------------------------------------------------------ init
__global__ void init_kernel(float* __restrict__ E, long ms, int n, int m, int l, int x_row0, int u_row0,
                            const float* __restrict__ X_k, const float* __restrict__ U_prev,
                            const float* __restrict__ W0)
{
    const int i = blockIdx.y;
    float* Ei = E + (long)i * ms;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (n + l) * m; e += gridDim.x * blockDim.x) {
        if (e < n * m) {
            Ei[(long)x_row0 * m + e] = X_k[e];
        } else {
            const int r = e - n * m;
            Ei[(long)u_row0 * m + r] = U_prev[r] + W0[(long)i * l * m + r];
        }
    }
}

__global__ void u_advance_kernel(float* __restrict__ E, long ms, int m, int l, int u_from, int u_to,
                                 const float* __restrict__ W)
{
    const int i = blockIdx.y;
    float* Ei = E + (long)i * ms;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * m; e += gridDim.x * blockDim.x)
        Ei[(long)u_to * m + e] = Ei[(long)u_from * m + e] + W[(long)i * l * m + e];
}

// ----------------------------------------------------------------- means
__global__ void means_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet act, RowSet obs,
                             ObsNoise V, float* __restrict__ meanE, float* __restrict__ meanY)
{
    const int R = act.count, p = obs.count;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (R + p) * m) return;
    const int a = idx / m, j = idx - a * m;
    const bool is_obs = a >= R;
    const int c = a - R;
    const long off = (long)(is_obs ? obs.rows[c] : act.rows[a]) * m + j;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int i = 0;
    for (; i + 4 <= N; i += 4) {
        float v0 = E[(long)i * ms + off], v1 = E[(long)(i + 1) * ms + off];
        float v2 = E[(long)(i + 2) * ms + off], v3 = E[(long)(i + 3) * ms + off];
        if (is_obs) {
            v0 += obs_noise(V, i, c, p, m, j);
            v1 += obs_noise(V, i + 1, c, p, m, j);
            v2 += obs_noise(V, i + 2, c, p, m, j);
            v3 += obs_noise(V, i + 3, c, p, m, j);
        }
        s0 += v0; s1 += v1; s2 += v2; s3 += v3;
    }
    for (; i < N; ++i) {
        float v = E[(long)i * ms + off];
        if (is_obs) v += obs_noise(V, i, c, p, m, j);
        s0 += v;
    }
    const float mean = ((s0 + s1) + (s2 + s3)) / (float)N;
    if (is_obs) meanY[c * m + j] = mean;
    else meanE[a * m + j] = mean;
}

// ------------------------------------------------------------ covariance
constexpr int CBM = 64, CBN = 64, CKC = 16;

// part[s][a][c] = sum_{i in split s} sum_j L[a](i,j) * A_Y[c](i,j), where
// L = [anomalies of the active rows (a < R); anomalies of Y (a >= R)].
__global__ void __launch_bounds__(256)
cov_partial_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V,
                   const float* __restrict__ meanE, const float* __restrict__ meanY,
                   float* __restrict__ part, int splits)
{
    __shared__ __align__(16) float As[CKC][CBM];
    __shared__ __align__(16) float Bs[CKC][CBN];
    const int R = act.count, p = obs.count, M = R + p;
    const int bm0 = blockIdx.x * CBM, bn0 = blockIdx.y * CBN, s = blockIdx.z;
    const int i0 = (int)((long)s * N / splits), i1 = (int)((long)(s + 1) * N / splits);
    const int t = threadIdx.x, tx = t % 16, ty = t / 16;
    const int lr = t / 4, lc = (t % 4) * 4;       // loader: row, first column of 4

    // loader rows
    const int a = bm0 + lr;
    const bool a_ok = a < M;
    const bool a_obs = a >= R;
    const long a_off = a_ok ? (long)(a_obs ? obs.rows[a - R] : act.rows[a]) * m : 0;
    const float* a_mean = a_ok ? (a_obs ? meanY + (long)(a - R) * m : meanE + (long)a * m) : nullptr;
    const int cb = bn0 + lr;
    const bool c_ok = cb < p;
    const long c_off = c_ok ? (long)obs.rows[cb] * m : 0;
    const float* c_mean = c_ok ? meanY + (long)cb * m : nullptr;

    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;

    for (int i = i0; i < i1; ++i) {
        const float* Ei = E + (long)i * ms;
        for (int j0 = 0; j0 < m; j0 += CKC) {
            const int j = j0 + lc;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (j < m) {
                if (a_ok) {
                    float4 x = *reinterpret_cast<const float4*>(Ei + a_off + j);
                    const float4 mu = *reinterpret_cast<const float4*>(a_mean + j);
                    if (a_obs) {
                        const float4 z = obs_noise4(V, i, a - R, p, m, j);
                        x.x += z.x; x.y += z.y; x.z += z.z; x.w += z.w;
                    }
                    va = make_float4(x.x - mu.x, x.y - mu.y, x.z - mu.z, x.w - mu.w);
                }
                if (c_ok) {
                    float4 y = *reinterpret_cast<const float4*>(Ei + c_off + j);
                    const float4 z = obs_noise4(V, i, cb, p, m, j);
                    const float4 mu = *reinterpret_cast<const float4*>(c_mean + j);
                    vb = make_float4(y.x + z.x - mu.x, y.y + z.y - mu.y, y.z + z.z - mu.z,
                                     y.w + z.w - mu.w);
                }
            }
            As[lc + 0][lr] = va.x; As[lc + 1][lr] = va.y; As[lc + 2][lr] = va.z; As[lc + 3][lr] = va.w;
            Bs[lc + 0][lr] = vb.x; Bs[lc + 1][lr] = vb.y; Bs[lc + 2][lr] = vb.z; Bs[lc + 3][lr] = vb.w;
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < CKC; ++kk) {
                const float4 x = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
                const float4 y = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
                const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xa[u], yb[v], acc[u][v]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int ar = bm0 + ty * 4 + u;
        if (ar >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int cc = bn0 + tx * 4 + v;
            if (cc < p) part[((long)s * M + ar) * p + cc] = acc[u][v];
        }
    }
}

__global__ void cov_reduce_kernel(const float* __restrict__ part, int splits, int rows, int p,
                                  double* __restrict__ C)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * p) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += (double)part[(long)k * rows * p + idx];
    C[idx] = s;
}

// ------------------------------------------------------------------ gain
constexpr int G_THREADS = 256;
constexpr int G_ROWS_PER_WARP = 2;
constexpr int G_ROWS_PER_CTA = (G_THREADS / 32) * G_ROWS_PER_WARP;
constexpr int G_KMAX = 8;                       // p <= 256

// Every CTA factors Cyy = L L^T in shared memory (FP32, right-looking, odd
// row stride so column walks are bank-conflict free), then each warp solves
// L L^T k = c for its rows c of Cxy: lane owns entries r = lane + 32 k, the
// pivot value is broadcast by shuffle.
__global__ void __launch_bounds__(G_THREADS)
gain_kernel(const double* __restrict__ C, int R, int p, float* __restrict__ K, int* __restrict__ status)
{
    extern __shared__ float A[];                 // p x ps
    __shared__ int bad;
    const int ps = p | 1;
    const int tid = threadIdx.x;
    const double* Cyy = C + (long)R * p;
    for (int e = tid; e < p * p; e += G_THREADS) A[(e / p) * ps + (e % p)] = (float)Cyy[e];
    if (tid == 0) bad = 0;
    for (int j = 0; j < p; ++j) {
        __syncthreads();
        const float d = A[j * ps + j];
        if (!(d > 0.f)) {
            if (tid == 0) bad = 1;
            break;
        }
        const float ljj = sqrtf(d);
        const float inv = 1.f / ljj;
        __syncthreads();
        for (int i = j + 1 + tid; i < p; i += G_THREADS) A[i * ps + j] *= inv;
        if (tid == 0) A[j * ps + j] = ljj;
        __syncthreads();
        const int cnt = p - j - 1;
        for (int e = tid; e < cnt * cnt; e += G_THREADS) {
            const int ii = j + 1 + e / cnt, kk = j + 1 + e % cnt;
            if (kk <= ii) A[ii * ps + kk] = fmaf(-A[ii * ps + j], A[kk * ps + j], A[ii * ps + kk]);
        }
    }
    __syncthreads();
    const int warp = tid / 32, lane = tid % 32;
    if (bad) {
        if (blockIdx.x == 0 && tid == 0) atomicExch(status, DEV_NOTSPD);
        for (int rr = 0; rr < G_ROWS_PER_WARP; ++rr) {
            const int a = blockIdx.x * G_ROWS_PER_CTA + warp * G_ROWS_PER_WARP + rr;
            if (a < R)
                for (int r = lane; r < p; r += 32) K[(long)a * p + r] = 0.f;
        }
        return;
    }
    for (int rr = 0; rr < G_ROWS_PER_WARP; ++rr) {
        const int a = blockIdx.x * G_ROWS_PER_CTA + warp * G_ROWS_PER_WARP + rr;
        if (a >= R) break;                       // warp-uniform
        float v[G_KMAX];
#pragma unroll
        for (int k = 0; k < G_KMAX; ++k) {
            const int r = lane + 32 * k;
            v[k] = (r < p) ? (float)C[(long)a * p + r] : 0.f;
        }
        // forward: L z = c
#pragma unroll
        for (int kb = 0; kb < G_KMAX; ++kb) {
            if (kb * 32 >= p) break;
            for (int il = 0; il < 32; ++il) {
                const int i = kb * 32 + il;
                if (i >= p) break;
                const float zi = __shfl_sync(0xffffffffu, v[kb], il) / A[i * ps + i];
                if (lane == il) v[kb] = zi;
#pragma unroll
                for (int k = 0; k < G_KMAX; ++k) {
                    if (k < kb) continue;
                    const int r = lane + 32 * k;
                    if (r > i && r < p) v[k] = fmaf(-A[r * ps + i], zi, v[k]);
                }
            }
        }
        // backward: L^T k = z
#pragma unroll
        for (int kb = G_KMAX - 1; kb >= 0; --kb) {
            if (kb * 32 >= p) continue;
            for (int il = 31; il >= 0; --il) {
                const int i = kb * 32 + il;
                if (i >= p) continue;
                const float ki = __shfl_sync(0xffffffffu, v[kb], il) / A[i * ps + i];
                if (lane == il) v[kb] = ki;
#pragma unroll
                for (int k = 0; k < G_KMAX; ++k) {
                    if (k > kb) continue;
                    const int r = lane + 32 * k;
                    if (r < i) v[k] = fmaf(-A[i * ps + r], ki, v[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < G_KMAX; ++k) {
            const int r = lane + 32 * k;
            if (r < p) K[(long)a * p + r] = v[k];
        }
    }
}

// ---------------------------------------------------------------- update
constexpr int U_CT = 64;     // columns per CTA
constexpr int U_RCH = 32;    // rows per K chunk

__global__ void __launch_bounds__(256)
update_kernel(float* __restrict__ E, long ms, int m, RowSet act, RowSet obs, ObsNoise V,
              const float* __restrict__ K, const float* __restrict__ Yx, const float* __restrict__ Yu,
              int n_yx)
{
    extern __shared__ __align__(16) float sm[];
    const int R = act.count, p = obs.count;
    float* D = sm;                               // [p][U_CT]
    float* Kt = sm + p * U_CT;                   // [p][U_RCH]
    const int i = blockIdx.x;
    const int j0 = blockIdx.y * U_CT;
    const int tid = threadIdx.x;
    float* Ei = E + (long)i * ms;

    // innovation D^i = Ybar - (H E^i + V^i), taken from the prior before any write
    for (int e = tid; e < p * U_CT; e += blockDim.x) {
        const int c = e / U_CT, jj = e - c * U_CT, j = j0 + jj;
        float d = 0.f;
        if (j < m) {
            const float yb = c < n_yx ? Yx[(long)c * m + j] : Yu[(long)(c - n_yx) * m + j];
            d = yb - (Ei[(long)obs.rows[c] * m + j] + obs_noise(V, i, c, p, m, j));
        }
        D[c * U_CT + jj] = d;
    }
    const int jj = tid % U_CT, rg = tid / U_CT;  // rg in 0..3, rows rg*8 .. rg*8+7 of a chunk
    const int j = j0 + jj;
    for (int a0 = 0; a0 < R; a0 += U_RCH) {
        __syncthreads();                         // D ready / previous chunk consumed
        for (int e = tid; e < p * U_RCH; e += blockDim.x) {
            const int c = e / U_RCH, rr = e - c * U_RCH;
            const int a = a0 + rr;
            Kt[c * U_RCH + rr] = a < R ? K[(long)a * p + c] : 0.f;
        }
        __syncthreads();
        float acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = 0.f;
        for (int c = 0; c < p; ++c) {
            const float d = D[c * U_CT + jj];
            const float4 k0 = *reinterpret_cast<const float4*>(&Kt[c * U_RCH + rg * 8]);
            const float4 k1 = *reinterpret_cast<const float4*>(&Kt[c * U_RCH + rg * 8 + 4]);
            acc[0] = fmaf(k0.x, d, acc[0]); acc[1] = fmaf(k0.y, d, acc[1]);
            acc[2] = fmaf(k0.z, d, acc[2]); acc[3] = fmaf(k0.w, d, acc[3]);
            acc[4] = fmaf(k1.x, d, acc[4]); acc[5] = fmaf(k1.y, d, acc[5]);
            acc[6] = fmaf(k1.z, d, acc[6]); acc[7] = fmaf(k1.w, d, acc[7]);
        }
        if (j < m) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int a = a0 + rg * 8 + q;
                if (a < R) Ei[(long)act.rows[a] * m + j] += acc[q];
            }
        }
    }
}

__global__ void block_means_kernel(const float* __restrict__ E, long ms, int N, int m, int row0,
                                   int rows_per_block, int n_blocks, float* __restrict__ out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_blocks * rows_per_block * m) return;
    const long off = (long)row0 * m + idx;      // blocks are contiguous rows
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int i = 0;
    for (; i + 4 <= N; i += 4) {
        s0 += E[(long)i * ms + off];
        s1 += E[(long)(i + 1) * ms + off];
        s2 += E[(long)(i + 2) * ms + off];
        s3 += E[(long)(i + 3) * ms + off];
    }
    for (; i < N; ++i) s0 += E[(long)i * ms + off];
    out[idx] = ((s0 + s1) + (s2 + s3)) / (float)N;
}

}  // namespace

void launch_ensemble_init(float* E, long ms, int N, int n, int m, int l, int x_row0, int u_row0, const float* X_k, const float* U_prev,
                          const float* W0, cudaStream_t st)
{
    dim3 grid(((n + l) * m + 255) / 256, N);
    init_kernel<<<grid, 256, 0, st>>>(E, ms, n, m, l, x_row0, u_row0, X_k, U_prev, W0);
}

void launch_u_advance(float* E, long ms, int N, int m, int l, int u_from, int u_to, const float* W,
                      cudaStream_t st)
{
    dim3 grid((l * m + 255) / 256, N);
    u_advance_kernel<<<grid, 256, 0, st>>>(E, ms, m, l, u_from, u_to, W);
}

void launch_means(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V,
                  float* meanE, float* meanY, cudaStream_t st)
{
    const int total = (act.count + obs.count) * m;
    means_kernel<<<(total + 255) / 256, 256, 0, st>>>(E, ms, N, m, act, obs, V, meanE, meanY);
}

int cov_splits(int R, int p, int N)
{
    const int tiles = ((R + p + CBM - 1) / CBM) * ((p + CBN - 1) / CBN);
    int s = (2 * 148 + tiles - 1) / tiles;
    if (s > N) s = N;
    if (s < 1) s = 1;
    return s;
}

void launch_cov_partial(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V,
                        const float* meanE, const float* meanY, float* part, int splits,
                        cudaStream_t st)
{
    const int M = act.count + obs.count, p = obs.count;
    dim3 grid((M + CBM - 1) / CBM, (p + CBN - 1) / CBN, splits);
    cov_partial_kernel<<<grid, 256, 0, st>>>(E, ms, N, m, act, obs, V, meanE, meanY, part, splits);
}

void launch_cov_reduce(const float* part, int splits, int rows, int p, double* C, cudaStream_t st)
{
    const int total = rows * p;
    cov_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(part, splits, rows, p, C);
}

size_t gain_smem_bytes(int p) { return sizeof(float) * (size_t)p * (size_t)(p | 1); }

void launch_gain(const double* C, int R, int p, float* K, int* status, cudaStream_t st)
{
    const size_t smem = gain_smem_bytes(p);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(gain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int grid = (R + G_ROWS_PER_CTA - 1) / G_ROWS_PER_CTA;
    gain_kernel<<<grid > 0 ? grid : 1, G_THREADS, smem, st>>>(C, R, p, K, status);
}

void launch_update(float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V,
                   const float* K, const float* Yx, const float* Yu, int n_yx, cudaStream_t st)
{
    const int p = obs.count;
    const size_t smem = sizeof(float) * (size_t)p * (U_CT + U_RCH);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    dim3 grid(N, (m + U_CT - 1) / U_CT);
    update_kernel<<<grid, 256, smem, st>>>(E, ms, m, act, obs, V, K, Yx, Yu, n_yx);
}

void launch_block_means(const float* E, long ms, int N, int m, int row0, int rows_per_block,
                        int n_blocks, float* out, cudaStream_t st)
{
    const int total = n_blocks * rows_per_block * m;
    block_means_kernel<<<(total + 255) / 256, 256, 0, st>>>(E, ms, N, m, row0, rows_per_block,
                                                            n_blocks, out);
}

}  // namespace oic
