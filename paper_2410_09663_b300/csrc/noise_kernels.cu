// noise_kernels.cu -- the random numbers Kalman-MPC draws (W0, W, V_X, V_U of
// Eq. (virtual-system) and Eq. (Ybar-samples)) generated on the device into
// the solve's noise buffer, for the paths that read them from memory; the
// generator itself (Philox-4x32-10 + Box-Muller) is philox.cuh.
#include "oic_internal.cuh"
#include "philox.cuh"

namespace oic {
namespace {

constexpr int MAX_SEG = 8;
struct Segs {
    unsigned long long end[MAX_SEG];
    float sigma[MAX_SEG];
    int n;
    int quad_ends;       // every end is a multiple of 4
};

__global__ void philox_noise_kernel(float* __restrict__ out, unsigned long long total,
                                    unsigned long long seed, const unsigned long long* __restrict__ solve_ctr,
                                    Segs segs)
{
    pdl_begin();
    const unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long e0 = q * 4ull;
    if (e0 >= total) return;
    float z[4];
    philox_normals4(seed, *solve_ctr, q, z);
    // sigma of each element's segment; the search is unrolled over the fixed
    // table size so the table stays in registers (a runtime index would put
    // it in local memory).  With every segment end a multiple of 4 (quad_ends)
    // the four elements share one segment and one search.
    float sg[4];
    const int nsearch = segs.quad_ends ? 1 : 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (t >= nsearch) {
            sg[t] = sg[0];
            continue;
        }
        const unsigned long long e = e0 + t;
        sg[t] = 0.f;
        bool found = false;
#pragma unroll
        for (int g = 0; g < MAX_SEG; ++g)
            if (!found && g < segs.n && e < segs.end[g]) {
                sg[t] = segs.sigma[g];
                found = true;
            }
    }
    if (e0 + 4 <= total && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        *reinterpret_cast<float4*>(out + e0) = make_float4(__fmul_rn(sg[0], z[0]), __fmul_rn(sg[1], z[1]),
                                                           __fmul_rn(sg[2], z[2]), __fmul_rn(sg[3], z[3]));
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (e0 + t < total) out[e0 + t] = __fmul_rn(sg[t], z[t]);
    }
}

// the solve index lives on the device, so a captured step graph draws fresh
// noise on every replay
__global__ void counter_tick_kernel(unsigned long long* ctr) {
    pdl_begin(); *ctr += 1ull; }

}  // namespace

void launch_philox_noise(float* out, size_t count_total, unsigned long long seed,
                         unsigned long long* solve_ctr, const size_t* seg_end, const float* seg_sigma,
                         int n_seg, cudaStream_t st, bool tick)
{
    Segs s{};
    s.n = n_seg < MAX_SEG ? n_seg : MAX_SEG;
    s.quad_ends = 1;
    for (int g = 0; g < s.n; ++g) {
        s.end[g] = seg_end[g];
        s.sigma[g] = seg_sigma[g];
        if (seg_end[g] % 4 != 0) s.quad_ends = 0;
    }
    const unsigned long long quads = (count_total + 3) / 4;
    const unsigned blocks = (unsigned)((quads + 255) / 256);
    pdl_launch(philox_noise_kernel, blocks, 256, 0, st, out, count_total, seed, solve_ctr, s);
    if (tick) pdl_launch(counter_tick_kernel, 1, 1, 0, st, solve_ctr);
}

}  // namespace oic
