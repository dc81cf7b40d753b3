// tc_tf32.cuh -- TF32 tensor-core building blocks shared by the
// covariance products and the member update: 128-byte-swizzled K-major
// operand tiles, the TF32 hi / lo split, 1-D bulk copies into shared memory
// and the tcgen05 MMA with TF32 operands.
#pragma once
#include <cstdint>

#include "tc_sm103.cuh"

namespace oic {
namespace tf32 {

// byte offset of (row r, 16-byte chunk k) in a 128-byte-swizzled K-major tile
__host__ __device__ __forceinline__ int swz(int r, int k) { return r * 128 + ((k ^ (r & 7)) << 4); }

// round to TF32 (10 stored mantissa bits), nearest with ties away from
// zero: add half an ulp of the kept part to the magnitude bits, clear the
// dropped 13 bits (a carry into the exponent is the correct rounding)
__device__ __forceinline__ float tf32_rna(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split_tf32(const float4& d, float4& hi, float4& lo)
{
    hi.x = tf32_rna(d.x); lo.x = tf32_rna(d.x - hi.x);
    hi.y = tf32_rna(d.y); lo.y = tf32_rna(d.y - hi.y);
    hi.z = tf32_rna(d.z); lo.z = tf32_rna(d.z - hi.z);
    hi.w = tf32_rna(d.w); lo.w = tf32_rna(d.w - hi.w);
}
__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 f4sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }

__device__ __forceinline__ void st_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void st_bulk(uint32_t dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(tc::smem_u32(mbar))
                 : "memory");
}
// K-major, 128-byte swizzle: SBO = 1024 B between 8-row groups, LBO unused
// (1), descriptor version bit 46, layout type 2 in bits 61-63.
constexpr uint32_t SW_DESC_HI = (1024u >> 4) | (1u << 14) | (2u << 29);
__device__ __forceinline__ uint32_t sw_desc(uint32_t saddr) { return ((saddr & 0x3FFFFu) >> 4) | (1u << 16); }
__device__ __forceinline__ void st_mma(uint32_t d, uint32_t a, uint32_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .b64 da, db;\n\t.reg .pred p;\n\t"
        "mov.b64 da, {%1, %5};\n\t"
        "mov.b64 db, {%2, %5};\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "r"(b), "r"(idesc), "r"(acc), "r"(SW_DESC_HI)
        : "memory");
}
// The same MMA called by a whole warp with warp-uniform operands: the
// elected lane issues it, and the operands stay in uniform registers.
__device__ __forceinline__ void st_mma_el(uint32_t d, uint32_t a, uint32_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .b64 da, db;\n\t.reg .pred p, e;\n\t"
        "mov.b64 da, {%1, %5};\n\t"
        "mov.b64 db, {%2, %5};\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "r"(b), "r"(idesc), "r"(acc), "r"(SW_DESC_HI)
        : "memory");
}
// instruction descriptor: TF32 A and B (format 2), FP32 D, K-major, N, M
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

}  // namespace tf32
}  // namespace oic
