// philox.cuh -- the device Philox stream of a solve's random numbers, as a
// generator every kernel can call: the noise kernel writes the stream to a
// buffer, and the kernels that consume it can instead draw their own
// elements in place (the same arithmetic, so the same values bit for bit).
//
// Generator: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit
// key, ten rounds of two 32 x 32 -> 64-bit multiplies whose high halves are
// xored with the other counter words and the key, with a Weyl increment of
// the key between rounds.  Element e of a solve's stream takes word e % 4 of
// the block for counter (e / 4 low, e / 4 high, solve low, solve high) under
// key (seed low, seed high).  Words become uniforms u = (w >> 8 + 1/2) 2^-24
// in (0, 1) (exact in float) and pairs become normals by Box-Muller:
// z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace oic {

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

// The four standard normals of counter block q of solve `solve`.
__device__ __forceinline__ void philox_normals4(unsigned long long seed, unsigned long long solve,
                                                unsigned long long q, float (&z)[4])
{
    const uint4 ctr = make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)solve, (uint32_t)(solve >> 32));
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 w = philox4x32_10(ctr, key);
    {
        const float r = sqrtf(-2.f * logf(word_to_uniform(w.x)));
        float s, c;
        sincospif(2.f * word_to_uniform(w.y), &s, &c);
        z[0] = __fmul_rn(r, c);
        z[1] = __fmul_rn(r, s);
    }
    {
        const float r = sqrtf(-2.f * logf(word_to_uniform(w.z)));
        float s, c;
        sincospif(2.f * word_to_uniform(w.w), &s, &c);
        z[2] = __fmul_rn(r, c);
        z[3] = __fmul_rn(r, s);
    }
}

// Where a kernel takes one segment of the solve's random numbers (W0, W_t,
// V_X,t, V_U,t, eps_t): element e of the segment is buf[e] when the buffer is
// materialised, else sigma * z[base + e] drawn in place from the stream of
// the solve index *ctr (base: the segment's first element in the stream,
// a multiple of 4).  Products are rounded on their own (__fmul_rn), as the
// buffer's values are, so a consumer's sum with them is the same either way.
struct NoiseSrc {
    const float* buf = nullptr;
    const unsigned long long* ctr = nullptr;
    unsigned long long seed = 0, base = 0;
    float sigma = 0.f;
    __host__ __device__ bool live() const { return buf != nullptr || ctr != nullptr; }
};

// Elements e .. e+3 (e % 4 == 0).
__device__ __forceinline__ float4 noise4(const NoiseSrc& s, long e)
{
    if (s.buf != nullptr) return *reinterpret_cast<const float4*>(s.buf + e);
    float z[4];
    philox_normals4(s.seed, *s.ctr, (s.base + (unsigned long long)e) >> 2, z);
    return make_float4(__fmul_rn(s.sigma, z[0]), __fmul_rn(s.sigma, z[1]), __fmul_rn(s.sigma, z[2]),
                       __fmul_rn(s.sigma, z[3]));
}

// Element e alone.
__device__ __forceinline__ float noise1(const NoiseSrc& s, long e)
{
    if (s.buf != nullptr) return s.buf[e];
    float z[4];
    const unsigned long long g = s.base + (unsigned long long)e;
    philox_normals4(s.seed, *s.ctr, g >> 2, z);
    const int t = (int)(g & 3ull);
    return __fmul_rn(s.sigma, t == 0 ? z[0] : t == 1 ? z[1] : t == 2 ? z[2] : z[3]);
}

}  // namespace oic
