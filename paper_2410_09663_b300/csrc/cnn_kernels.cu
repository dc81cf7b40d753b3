// cnn_kernels.cu -- the CNN surrogate X_{t+1} = CNN_theta(X_t, U_t) of Eq. (1)
// on CUDA cores (FP32 FFMA), used for the ensemble rollout of
// Eq. (prediction-samplewise) and for the plant step of Algorithm 1.
//
// Activations are channel-planar per member: act[b][c][y][x].  A 3x3 "same"
// layer is a direct convolution over a 16 x 16 output tile per CTA with the
// (16 + 2)^2 input halo staged in shared memory, CI_T input channels at a
// time; every thread owns one output pixel and CO_T output channels.
#include "oic_internal.cuh"

namespace oic {
namespace {

constexpr int TILE = 16;
constexpr int HALO = TILE + 2;
constexpr int CI_T = 8;

// act0[b][0] = X^b, act0[b][1] = B U^b   (Eq. (1) input [X; B U]).
__global__ void cnn_input_kernel(const float* __restrict__ X, long x_ms, const float* __restrict__ U,
                                 long u_ms, const float* __restrict__ B, float* __restrict__ act0,
                                 int n, int m, int l)
{
    pdl_begin();
    const int b = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * m) return;
    const int y = idx / m, x = idx - y * m;
    const float* Xb = X + (long)b * x_ms;
    const float* Ub = U + (long)b * u_ms;
    float s = 0.f;
    for (int c = 0; c < l; ++c) s = fmaf(B[y * l + c], Ub[c * m + x], s);
    float* a = act0 + (long)b * 2 * n * m;
    a[idx] = Xb[idx];
    a[n * m + idx] = s;
}

// MODE 0: out = tanh(conv + bias) for CO_T channels starting at blockIdx.y*CO_T.
// MODE 1: Cout = 1, out = xres + rs * (conv + bias)  (last layer + residual).
template <int CO_T, int MODE>
__global__ void __launch_bounds__(TILE * TILE)
conv3x3_kernel(const float* __restrict__ in, int Cin, float* __restrict__ out, long out_ms, int Cout,
               int n, int m, const float* __restrict__ w, const float* __restrict__ bias,
               const float* __restrict__ xres, long xres_ms, float rs)
{
    pdl_begin();
    __shared__ float tile[CI_T][HALO][HALO + 1];
    __shared__ float ws[CO_T][CI_T * 9];

    const int tiles_x = (m + TILE - 1) / TILE;
    const int tx0 = (blockIdx.x % tiles_x) * TILE;
    const int ty0 = (blockIdx.x / tiles_x) * TILE;
    const int co0 = blockIdx.y * CO_T;
    const int b = blockIdx.z;
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    const float* inb = in + (long)b * Cin * n * m;

    float acc[CO_T];
#pragma unroll
    for (int k = 0; k < CO_T; ++k) acc[k] = 0.f;

    for (int ci0 = 0; ci0 < Cin; ci0 += CI_T) {
        for (int e = threadIdx.x; e < CI_T * HALO * HALO; e += TILE * TILE) {
            const int c = e / (HALO * HALO);
            const int r = e - c * HALO * HALO;
            const int yy = ty0 - 1 + r / HALO, xx = tx0 - 1 + r % HALO;
            float v = 0.f;
            if (ci0 + c < Cin && yy >= 0 && yy < n && xx >= 0 && xx < m)
                v = inb[((long)(ci0 + c) * n + yy) * m + xx];
            tile[c][r / HALO][r % HALO] = v;
        }
        for (int e = threadIdx.x; e < CO_T * CI_T * 9; e += TILE * TILE) {
            const int k = e / (CI_T * 9);
            const int r = e - k * CI_T * 9;
            const int c = r / 9, tap = r - c * 9;
            float v = 0.f;
            if (co0 + k < Cout && ci0 + c < Cin) v = w[((long)(co0 + k) * Cin + ci0 + c) * 9 + tap];
            ws[k][r] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < CI_T; ++c) {
            float v[9];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) v[dy * 3 + dx] = tile[c][ty + dy][tx + dx];
#pragma unroll
            for (int k = 0; k < CO_T; ++k)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[k] = fmaf(ws[k][c * 9 + t], v[t], acc[k]);
        }
        __syncthreads();
    }

    const int y = ty0 + ty, x = tx0 + tx;
    if (y >= n || x >= m) return;
    if (MODE == 0) {
        float* ob = out + (long)b * Cout * n * m;
#pragma unroll
        for (int k = 0; k < CO_T; ++k)
            if (co0 + k < Cout) ob[((long)(co0 + k) * n + y) * m + x] = tanhf(acc[k] + bias[co0 + k]);
    } else {
        const float xv = xres[(long)b * xres_ms + y * m + x];
        out[(long)b * out_ms + y * m + x] = fmaf(rs, acc[0] + bias[0], xv);
    }
}

}  // namespace

void launch_cnn_input(const float* X, long x_ms, const float* U, long u_ms, const float* B,
                      float* act0, int Nb, int n, int m, int l, cudaStream_t st)
{
    dim3 grid((n * m + 255) / 256, Nb);
    pdl_launch(cnn_input_kernel, grid, 256, 0, st, X, x_ms, U, u_ms, B, act0, n, m, l);
}

void launch_conv_hidden(const float* in, int Cin, float* out, int Cout, int Nb, int n, int m,
                        const float* w, const float* bias, cudaStream_t st)
{
    const int tiles = ((m + TILE - 1) / TILE) * ((n + TILE - 1) / TILE);
    constexpr int CO = 16;
    dim3 grid(tiles, (Cout + CO - 1) / CO, Nb);
    pdl_launch(conv3x3_kernel<CO, 0>, grid, TILE * TILE, 0, st, in, Cin, out, 0, Cout, n, m, w, bias,
                                                        nullptr, 0, 0.f);
}

void launch_conv_out_residual(const float* in, int Cin, const float* Xin, long xin_ms, float* Xout,
                              long xout_ms, int Nb, int n, int m, const float* w,
                              const float* bias, float rs, cudaStream_t st)
{
    const int tiles = ((m + TILE - 1) / TILE) * ((n + TILE - 1) / TILE);
    dim3 grid(tiles, 1, Nb);
    pdl_launch(conv3x3_kernel<1, 1>, grid, TILE * TILE, 0, st, in, Cin, Xout, xout_ms, 1, n, m, w, bias,
                                                       Xin, xin_ms, rs);
}

}  // namespace oic
