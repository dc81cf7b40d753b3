// control_transform.cu -- the right transformation for narrow controls (the
// paragraph after the paper's Table I): U = u T widens a control u of mu < m
// columns for the matrix-variate method, and u = U T^T (T T^T)^{-1} maps a
// smoothed U back.
#include "oic_internal.cuh"

namespace oic {
namespace {

__device__ int g_ctl_status;                            // 0, or pivot + 1 where T T^T is not SPD

// U[r][j] = sum_c u[r][c] T[c][j]: one thread per element.
__global__ void control_expand_kernel(const float* __restrict__ u, int l, int mu, const float* __restrict__ T, int m,
                                      float* __restrict__ U)
{
    pdl_begin();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= l * m) return;
    const int r = e / m, j = e % m;
    float s = 0.f;
    for (int c = 0; c < mu; ++c) s = fmaf(u[r * mu + c], T[(long)c * m + j], s);
    U[e] = s;
}

// One CTA: G = T T^T and W = U T^T in FP64 (shared memory), G = L L^T
// (right-looking, one pivot per barrier), then each thread takes rows r of W
// and solves L z = w_r, L^T u_r = z.
constexpr int CT_T = 256;

__global__ void __launch_bounds__(CT_T)
control_reduce_kernel(const float* __restrict__ U, int l, int m, const float* __restrict__ T, int mu,
                      float* __restrict__ u)
{
    pdl_begin();
    extern __shared__ double cs[];
    double* G = cs;                                     // [mu][mu], then L (lower)
    double* W = cs + mu * mu;                           // [l][mu]
    __shared__ int bad;
    const int tid = threadIdx.x;
    for (int e = tid; e < mu * mu; e += CT_T) {
        const int a = e / mu, b = e % mu;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma((double)T[(long)a * m + j], (double)T[(long)b * m + j], s);
        G[e] = s;
    }
    for (int e = tid; e < l * mu; e += CT_T) {
        const int r = e / mu, a = e % mu;
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma((double)U[(long)r * m + j], (double)T[(long)a * m + j], s);
        W[e] = s;
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < mu; ++j) {
        const double d = G[j * mu + j];
        if (!(d > 0.0)) {                               // the same value in every thread
            if (tid == 0) bad = j + 1;
            break;
        }
        const double ljj = sqrt(d);
        __syncthreads();
        for (int i = j + 1 + tid; i < mu; i += CT_T) G[i * mu + j] /= ljj;
        __syncthreads();
        for (int e = tid; e < (mu - j - 1) * (mu - j - 1); e += CT_T) {
            const int i = j + 1 + e / (mu - j - 1), k = j + 1 + e % (mu - j - 1);
            if (k <= i) G[i * mu + k] = fma(-G[i * mu + j], G[k * mu + j], G[i * mu + k]);
        }
        if (tid == 0) G[j * mu + j] = ljj;
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) g_ctl_status = bad;
    if (bad) return;
    for (int r = tid; r < l; r += CT_T) {
        double* w = W + r * mu;
        for (int i = 0; i < mu; ++i) {                  // L z = w (z over w)
            double s = w[i];
            for (int k = 0; k < i; ++k) s = fma(-G[i * mu + k], w[k], s);
            w[i] = s / G[i * mu + i];
        }
        for (int i = mu - 1; i >= 0; --i) {             // L^T u_r = z
            double s = w[i];
            for (int k = i + 1; k < mu; ++k) s = fma(-G[k * mu + i], w[k], s);
            w[i] = s / G[i * mu + i];
        }
        for (int i = 0; i < mu; ++i) u[r * mu + i] = (float)w[i];
    }
}

}  // namespace

extern "C" oic_status oic_control_expand(const float* u, int l, int mu, const float* T, int m, float* U,
                                         void* cuda_stream)
{
    if (!u || !T || !U || mu < 1 || mu > m || m > 1024 || l < 1 || l > 4096) return OIC_EINVAL;
    const int n = l * m;
    pdl_launch(control_expand_kernel, (n + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream), u, l, mu, T, m,
               U);
    return cudaGetLastError() == cudaSuccess ? OIC_OK : OIC_ECUDA;
}

extern "C" oic_status oic_control_reduce(const float* U, int l, int m, const float* T, int mu, float* u,
                                         void* cuda_stream)
{
    if (!U || !T || !u || mu < 1 || mu > 64 || mu > m || m > 1024 || l < 1 || l > 256) return OIC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t smem = sizeof(double) * ((size_t)mu * mu + (size_t)l * mu);
    static DeviceOnce attr_set;
    if (!attr_set.run([] {
            return cudaFuncSetAttribute(control_reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(double) * (64 * 64 + 256 * 64))) == cudaSuccess;
        }))
        return OIC_ECUDA;
    pdl_launch(control_reduce_kernel, 1, CT_T, smem, st, U, l, m, T, mu, u);
    int status = 0;
    if (cudaMemcpyFromSymbolAsync(&status, g_ctl_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return OIC_ECUDA;
    return status ? OIC_ENOTSPD : OIC_OK;
}

}  // namespace oic
