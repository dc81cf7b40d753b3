// constraint_obs.cu -- virtual observations of state/input constraints (the
// paragraph on constraints after Table I of arXiv 2410.09663).
//
// A constraint g(X, U) <= 0 is observed as z = phi(g(X_t, U_t)) + eps with
// reference 0 and the softplus barrier phi(x) = ln(1 + e^{beta x}) / alpha.
// Each of the c constraints is one row of m values, affine per column in the
// member's predicted field and control:
//     g[r][j] = sum_a Gx[r][a] X_t[a][j] + sum_b Gu[r][b] U_t[b][j] - h[r].
// The rows are written into the member's constraint block of the ensemble,
// after which the covariance and update kernels treat them as plain observed
// rows (noise already added, reference 0).
//
// Work: N c m (nk + O(1)) flops and N (nk + c) m floats of traffic per
// assimilation time (nk = columns of [Gx Gu] that are not all zero, l for a
// box on U); a few microseconds at 64 x 64, N = 256.
#include "oic_internal.cuh"

namespace oic {
namespace {

// ln(1 + e^y) as max(y, 0) + log1p(e^{-|y|}): the same function, and e^{-|y|}
// cannot overflow.
__device__ __forceinline__ float softplus_barrier(float x, float alpha, float beta)
{
    const float y = beta * x;
    return (fmaxf(y, 0.f) + log1pf(expf(-fabsf(y)))) / alpha;
}

// Thread unit: (member i, constraint row r, 4 consecutive columns j).
__global__ void __launch_bounds__(256)
constraint_obs_kernel(float* __restrict__ E, long ms, int N, int m, int n, int xrow, int urow, int zrow, int c,
                      const float* __restrict__ G, const int* __restrict__ cols, int nk,
                      const float* __restrict__ h, float alpha, float beta, NoiseSrc eps)
{
    pdl_begin();
    const int m4 = m / 4;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)N * c * m4) return;
    const int j = 4 * (int)(e % m4);
    const int r = (int)((e / m4) % c);
    const int i = (int)(e / ((long)m4 * c));
    float* Ei = E + (long)i * ms;
    const float hr = h[r];
    float4 g = make_float4(-hr, -hr, -hr, -hr);
#pragma unroll 8
    for (int k = 0; k < nk; ++k) {                   // unrolled: the row loads issue together
        const int a = cols[k];
        const int row = a < n ? xrow + a : urow + (a - n);
        const float w = G[(long)r * nk + k];
        const float4 v = *reinterpret_cast<const float4*>(Ei + (long)row * m + j);
        g.x = fmaf(w, v.x, g.x);
        g.y = fmaf(w, v.y, g.y);
        g.z = fmaf(w, v.z, g.z);
        g.w = fmaf(w, v.w, g.w);
    }
    float4 z = make_float4(softplus_barrier(g.x, alpha, beta), softplus_barrier(g.y, alpha, beta),
                           softplus_barrier(g.z, alpha, beta), softplus_barrier(g.w, alpha, beta));
    if (eps.live()) {
        const float4 v = noise4(eps, ((long)i * c + r) * m + j);
        z.x += v.x;
        z.y += v.y;
        z.z += v.z;
        z.w += v.w;
    }
    *reinterpret_cast<float4*>(Ei + (long)(zrow + r) * m + j) = z;
}

}  // namespace

void launch_constraint_obs(float* E, long ms, int N, int m, int n, int xrow, int urow, int zrow, int c,
                           const float* G, const int* cols, int nk, const float* h, float alpha, float beta,
                           NoiseSrc eps, cudaStream_t st)
{
    const long units = (long)N * c * (m / 4);
    const unsigned blocks = (unsigned)((units + 255) / 256);
    pdl_launch(constraint_obs_kernel, blocks, 256, 0, st, E, ms, N, m, n, xrow, urow, zrow, c, G, cols, nk, h,
               alpha, beta, eps);
}

}  // namespace oic
