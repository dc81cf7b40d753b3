// noise_kernels.cu -- the random numbers Kalman-MPC draws (W0, W, V_X, V_U of
// Eq. (virtual-system) and Eq. (Ybar-samples)) generated on the device.
//
// Generator: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit
// key, ten rounds of two 32 x 32 -> 64-bit multiplies whose high halves are
// xored with the other counter words and the key, with a Weyl increment of
// the key between rounds.  Element e of a solve's noise buffer takes word
// e % 4 of the block for counter (e / 4 low, e / 4 high, solve low, solve high)
// under key (seed low, seed high).  Words become uniforms u = (w >> 8 + 1/2)
// 2^-24 in (0, 1) (exact in float) and pairs become normals by Box-Muller:
// z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1).
#include "oic_internal.cuh"

namespace oic {
namespace {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = PHILOX_M0 * c.x, hi0 = __umulhi(PHILOX_M0, c.x);
        const uint32_t lo1 = PHILOX_M1 * c.z, hi1 = __umulhi(PHILOX_M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += PHILOX_W0;
        k.y += PHILOX_W1;
    }
    return c;
}

__device__ __forceinline__ float word_to_uniform(uint32_t w)
{
    return ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

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
    const unsigned long long solve = *solve_ctr;
    const uint4 ctr = make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)solve,
                                 (uint32_t)(solve >> 32));
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 w = philox4x32_10(ctr, key);
    float z[4];
    {
        const float r = sqrtf(-2.f * logf(word_to_uniform(w.x)));
        float s, c;
        sincospif(2.f * word_to_uniform(w.y), &s, &c);
        z[0] = r * c;
        z[1] = r * s;
    }
    {
        const float r = sqrtf(-2.f * logf(word_to_uniform(w.z)));
        float s, c;
        sincospif(2.f * word_to_uniform(w.w), &s, &c);
        z[2] = r * c;
        z[3] = r * s;
    }
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
        *reinterpret_cast<float4*>(out + e0) = make_float4(sg[0] * z[0], sg[1] * z[1], sg[2] * z[2], sg[3] * z[3]);
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (e0 + t < total) out[e0 + t] = sg[t] * z[t];
    }
}

// the solve index lives on the device, so a captured step graph draws fresh
// noise on every replay
__global__ void counter_tick_kernel(unsigned long long* ctr) {
    pdl_begin(); *ctr += 1ull; }

}  // namespace

void launch_philox_noise(float* out, size_t count_total, unsigned long long seed,
                         unsigned long long* solve_ctr, const size_t* seg_end, const float* seg_sigma,
                         int n_seg, cudaStream_t st)
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
    pdl_launch(counter_tick_kernel, 1, 1, 0, st, solve_ctr);
}

}  // namespace oic
