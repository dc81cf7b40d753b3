// cnn_fused_tc.cu -- the whole surrogate X_{t+1} = X_t + s * CNN_theta(X_t, U_t)
// of Eq. (1), structure [X; B U] -> C (tanh) -> C (tanh) -> 1, in ONE kernel,
// every layer on the tcgen05 tensor cores at FP32 accuracy:
//
//   operands are split x = hi + lo * 2^-11 (hi, lo fp16) and each layer
//   accumulates main = A_hi B_hi and corr = A_hi B_lo + A_lo B_hi in tensor
//   memory (out = main + corr * 2^-11, error ~2^-21 per product);
//   first layer (2 -> C)   K = 16 per horizontal tap holds [X, B U] of the
//                          three stencil rows, hi in one half and lo in the
//                          other; one N = 2C MMA per tap gives main and corr
//   hidden layer (C -> C)  K = C per tap; [B_hi; B_lo] stacked as N = 2C, then
//                          A_lo B_hi with N = C
//   last layer (C -> 1)    N = 16 columns hold main and corr of the three
//                          stencil rows; the CUDA cores turn them into rolling
//                          per-pixel sums over output rows r+1, r, r-1
//
// Only X, U and the weights are read and X_next written.  A CTA owns a group
// of G = 128/m members; an M = 128 tile is one image row of the group with
// the members INTERLEAVED pixel by pixel (position G + G x + b for member b,
// pixel x, zero pads at both ends), so a horizontal stencil tap is a shift of
// the operand start by G positions = 16 G bytes and one copy of each row
// serves all three taps.  Per hidden row r the tensor core runs first-layer
// row r+2, hidden row r and last layer of row r-1 while the CUDA cores drain
// the previous results (tanh, split, stores).  The grid is persistent over
// contiguous (group, row) ranges.
#include <cuda_fp16.h>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int FT = 544;                                 // 16 drain warps + 1 MMA-issuing warp
constexpr int ND = 512;                                 // drain threads
constexpr int FM = 128;                                 // tile rows (pixels)
constexpr int BAR_DRAIN = 1;                            // named barrier of the drain warps
constexpr long long F_WAIT = 4000000000LL;

__host__ __device__ constexpr int al16(int x) { return (x + 15) / 16 * 16; }

template <int C, int G>
struct FS {
    static constexpr int KC = C / 8, KS = C / 16;
    static constexpr int NPOS = FM + 2 * G;             // operand positions incl. pads
    static constexpr int PLANE = NPOS * 16;             // one (part, 8-channel) plane
    static constexpr int SLOT = 2 * KC * PLANE;         // hi and lo of one activation row
    static constexpr int FBUF = 2 * PLANE;              // first-layer operand: hi | lo
    static constexpr int BTILE = 2 * (2 * C) * 16;      // hidden (tap, K-step) tile
    static constexpr int BBYTES = 9 * KS * BTILE;
    static constexpr int B1BYTES = 3 * 2 * 64 * 16;     // first layer: 3 taps x (2 x 64 x 8)
    static constexpr int B3TILE = 2 * 16 * 16;          // last layer tile: 2 x 16 x 8
    static constexpr int B3BYTES = 3 * KS * 2 * B3TILE;
    static constexpr int NH1 = 4, NXB = 10;
    static constexpr int SP = NPOS | 1;                 // odd FP32 row stride
    static constexpr int OFF_H1 = 0;
    static constexpr int OFF_Z = OFF_H1 + NH1 * SLOT;   // permanently zero activation row
    static constexpr int OFF_H2 = OFF_Z + SLOT;
    static constexpr int OFF_F = OFF_H2 + 2 * SLOT;
    static constexpr int OFF_B = OFF_F + 2 * FBUF;
    static constexpr int OFF_B1 = OFF_B + BBYTES;
    static constexpr int OFF_B3 = OFF_B1 + B1BYTES;
    static constexpr int OFF_XB = OFF_B3 + B3BYTES;                    // [NXB][2][SP] fp32
    static constexpr int OFF_BIAS = OFF_XB + al16(NXB * 2 * SP * 4);   // b1[C], b2[C], b3
    static constexpr int OFF_MISC = OFF_BIAS + al16((2 * C + 4) * 4);  // mbarriers, TMEM base
    static constexpr int OFF_DYN = OFF_MISC + 128;                     // U group, B matrix
    static constexpr int ZERO_BYTES = OFF_B;                           // operand buffers incl. pads
    // tensor memory: first-layer, hidden and last-layer accumulators, double buffered
    static constexpr int T_F = 0, T_H = 4 * C, T_L = 8 * C;
    static constexpr int TMEM_COLS = 512;
};

__device__ __forceinline__ int mod_pos(int r, int k) { return ((r % k) + k) % k; }

// tanh(x) = 1 - 2 / (1 + e^{2x}): saturates correctly at both ends; absolute
// error a few 1e-7 (the exponential and the quotient are each within a few
// ulps), which is below the FP32 rounding of the layer's inputs.
__device__ __forceinline__ float tanh_fast(float x)
{
    return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x));
}

// 8 x 32-bit TMEM columns for the warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int C, int G>
__device__ __forceinline__ void issue_first(uint32_t s0, uint32_t acc, int r1)
{
    using S = FS<C, G>;
    constexpr uint32_t id = tc::idesc_f16(FM, 64);
    const uint32_t f = s0 + S::OFF_F + (r1 & 1) * S::FBUF;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
        const uint64_t da = tc::desc_kmajor(f + dx * G * 16, S::PLANE, 128);
        const uint64_t db = tc::desc_kmajor(s0 + S::OFF_B1 + dx * 2048, 64 * 16, 128);
        tc::mma_f16(acc, da, db, id, dx > 0 ? 1u : 0u);
    }
}

// Hidden row r from first-layer rows r-1, r, r+1; rows outside the image read
// the zero slot.
template <int C, int G>
__device__ __forceinline__ void issue_hidden(uint32_t s0, uint32_t acc, int r, int n)
{
    using S = FS<C, G>;
    constexpr uint32_t id1 = tc::idesc_f16(FM, 2 * C);
    constexpr uint32_t id2 = tc::idesc_f16(FM, C);
    uint32_t accumulate = 0;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const int j = r + dy - 1;
        const uint32_t slot = s0 + ((j < 0 || j >= n) ? S::OFF_Z : S::OFF_H1 + mod_pos(j, S::NH1) * S::SLOT);
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                const uint32_t a_hi = slot + (2 * ks) * S::PLANE + dx * G * 16;
                const uint32_t a_lo = slot + (S::KC + 2 * ks) * S::PLANE + dx * G * 16;
                const uint32_t b = s0 + S::OFF_B + ((dy * 3 + dx) * S::KS + ks) * S::BTILE;
                const uint64_t db = tc::desc_kmajor(b, 2 * C * 16, 128);
                tc::mma_f16(acc, tc::desc_kmajor(a_hi, S::PLANE, 128), db, id1, accumulate);
                tc::mma_f16(acc + C, tc::desc_kmajor(a_lo, S::PLANE, 128), db, id2, 1u);
                accumulate = 1;
            }
        }
    }
}

template <int C, int G>
__device__ __forceinline__ void issue_last(uint32_t s0, uint32_t acc, int h)
{
    using S = FS<C, G>;
    constexpr uint32_t id = tc::idesc_f16(FM, 16);
    const uint32_t buf = s0 + S::OFF_H2 + (h & 1) * S::SLOT;
    uint32_t accumulate = 0;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
        for (int ks = 0; ks < S::KS; ++ks) {
            const uint32_t a_hi = buf + (2 * ks) * S::PLANE + dx * G * 16;
            const uint32_t a_lo = buf + (S::KC + 2 * ks) * S::PLANE + dx * G * 16;
            const uint32_t b = s0 + S::OFF_B3 + (dx * S::KS + ks) * 2 * S::B3TILE;
            tc::mma_f16(acc, tc::desc_kmajor(a_hi, S::PLANE, 128), tc::desc_kmajor(b, 16 * 16, 128), id, accumulate);
            tc::mma_f16(acc, tc::desc_kmajor(a_lo, S::PLANE, 128), tc::desc_kmajor(b + S::B3TILE, 16 * 16, 128), id, 1u);
            accumulate = 1;
        }
    }
}

// mbarriers in the MISC region (8 bytes each)
enum : int {
    MB_F = 0,          // first layer done (tensor core -> drain warps)
    MB_H = 1,          // [2] hidden layer done, by row parity
    MB_L = 3,          // [2] last layer done, by row parity
    MB_RH1 = 5,        // first-layer row drained into its operand slot (16 warps)
    MB_RF = 6,         // [2] first-layer operand built, by row parity (4 warps)
    MB_RH2 = 8,        // [2] hidden row drained into its operand buffer (16 warps)
    MB_FIN = 10,       // every MMA of the kernel done
    MB_COUNT = 11
};

template <int C, int G>
__global__ void __launch_bounds__(FT, 1)
cnn_fused_kernel(const float* __restrict__ X, long x_ms, const float* __restrict__ U, long u_ms,
                 float* __restrict__ Xout, long o_ms, const float* __restrict__ Bmat, int Nb, int n, int l,
                 const float* __restrict__ b1, const __half* __restrict__ wpk2, const float* __restrict__ b2,
                 const __half* __restrict__ wpk13, const float* __restrict__ b3, float rs, int* __restrict__ err)
{
    using S = FS<C, G>;
    static_assert(C == 32, "16 drain warps = 4 lane quarters x 4 groups of 8 channels");
    static_assert(MB_COUNT * 8 + 4 <= 128, "MISC region");
    constexpr int m = FM / G;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* xb = reinterpret_cast<float*>(smem + S::OFF_XB);
    float* sbias = reinterpret_cast<float*>(smem + S::OFF_BIAS);   // b1 | b2 | b3
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + S::OFF_MISC);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::OFF_MISC + MB_COUNT * 8);
    float* su = reinterpret_cast<float*>(smem + S::OFF_DYN);                 // [G][l][m]
    float* sB = su + G * l * m;                                              // [n][l]
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t s0 = tc::smem_u32(smem);

    // ---- one-time set-up: zero the operand buffers (pads and the zero slot
    // stay zero), copy weights
    for (int e = tid; e < S::ZERO_BYTES / 16; e += FT)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < S::BBYTES / 16; e += FT)
        reinterpret_cast<uint4*>(smem + S::OFF_B)[e] = reinterpret_cast<const uint4*>(wpk2)[e];
    for (int e = tid; e < (S::B1BYTES + S::B3BYTES) / 16; e += FT)
        reinterpret_cast<uint4*>(smem + S::OFF_B1)[e] = reinterpret_cast<const uint4*>(wpk13)[e];
    for (int e = tid; e < S::NXB * 2 * S::SP; e += FT) xb[e] = 0.f;
    for (int e = tid; e < C; e += FT) { sbias[e] = b1[e]; sbias[C + e] = b2[e]; }
    for (int e = tid; e < n * l; e += FT) sB[e] = Bmat[e];
    if (tid == 0) {
        sbias[2 * C] = b3[0];
        for (int i = 0; i < MB_COUNT; ++i) {
            const int cnt = (i == MB_RH1 || i == MB_RH2 || i == MB_RH2 + 1) ? 16
                          : (i == MB_RF || i == MB_RF + 1) ? 4 : 1;
            tc::mbar_init(mb + i, cnt);
        }
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_holder, S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    const int groups = (Nb + G - 1) / G;
    const long total = (long)groups * n;
    const long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    uint32_t ph = 0;                                    // this thread's phase bit per mbarrier
    bool failed = false;
    auto wait = [&](int i) {
        if (!tc::mbar_wait_bounded(mb + i, (ph >> i) & 1u, F_WAIT)) {
            failed = true;
            atomicExch(err, DEV_TIMEOUT);
        }
        ph ^= 1u << i;
        tc::fence_after_sync();
    };
    const int q4 = warp & 3, cg = (warp >> 2) & 3;     // drain: lane quarter, channel group
    const int ep = 32 * q4 + lane;                      // drain pixel (TMEM lane)
    const uint32_t tlane = (uint32_t)(32 * q4) << 16;

    for (long t = t0; t < t1;) {
        const int g = (int)(t / n);
        const int ys = (int)(t % n);
        const long rem = t1 - t;
        const int ye = (long)(n - ys) < rem ? n : (int)(ys + rem);
        t += ye - ys;
        // output rows ys .. ye-1 need hidden rows r_lo .. r_hi and first-layer
        // rows r_lo-1 .. r_hi+1 (those inside the image are computed)
        const int r_lo = ys > 0 ? ys - 1 : 0;
        const int r_hi = ye < n ? ye : n - 1;
        const int f_lo = r_lo - 1 > 0 ? r_lo - 1 : 0;
        const int f_hi = r_hi + 1 < n - 1 ? r_hi + 1 : n - 1;
        auto Fvalid = [&](int f) { return f >= f_lo && f <= f_hi; };

        if (warp == ND / 32) {
            // ================= MMA-issuing warp (one thread) =================
            // iteration k: first-layer row k+3, hidden row k+1, last layer of row k
            if (lane == 0) {
                for (int k = r_lo - 4; k <= r_hi && !failed; ++k) {
                    if (Fvalid(k + 2)) wait(MB_RH1);                // rows k .. k+2 in their slots
                    const bool f3 = Fvalid(k + 3);
                    if (f3) wait(MB_RF + ((k + 3) & 1));           // operand of first-layer row k+3
                    if (f3) {
                        issue_first<C, G>(s0, tmem + S::T_F + ((k + 3) & 1) * 64, k + 3);
                        tc::mma_commit(mb + MB_F);
                    }
                    if (k + 1 >= r_lo && k + 1 <= r_hi) {
                        issue_hidden<C, G>(s0, tmem + S::T_H + ((k + 1) & 1) * 64, k + 1, n);
                        tc::mma_commit(mb + MB_H + ((k + 1) & 1));
                    }
                    if (k >= r_lo) {
                        wait(MB_RH2 + (k & 1));                     // hidden row k in its buffer
                        issue_last<C, G>(s0, tmem + S::T_L + (k & 1) * 16, k);
                        tc::mma_commit(mb + MB_L + (k & 1));
                    }
                }
            }
            __syncwarp();
        } else {
            // ================= 16 drain warps =================
            for (int e = tid; e < G * l * m; e += ND) {
                const int b = e / (l * m), rr = e % (l * m);
                const int mbr = g * G + b;
                su[e] = mbr < Nb ? U[(long)mbr * u_ms + rr] : 0.f;
            }
            tc::named_bar(BAR_DRAIN, ND);

            // [X; B U] row r into its ring slot (zero outside the image / group);
            // warps 8-11, the X row fetched one row ahead
            const bool xb_role = tid >= 2 * FM && tid < 3 * FM;
            const int xt = tid - 2 * FM;
            const int xb_b = xb_role ? xt / m : 0, xb_x = xb_role ? xt % m : 0;
            const int xb_mb = g * G + xb_b;
            auto fetch_x = [&](int r) -> float {
                return (xb_role && r >= 0 && r < n && xb_mb < Nb) ? X[(long)xb_mb * x_ms + (long)r * m + xb_x] : 0.f;
            };
            auto store_xb = [&](int r, float xv) {
                if (xb_role) {
                    float* d = xb + mod_pos(r, S::NXB) * 2 * S::SP;
                    const int q = G + G * xb_x + xb_b;
                    float bu = 0.f;
                    if (r >= 0 && r < n && xb_mb < Nb) {
                        const float* ub = su + xb_b * l * m + xb_x;
                        for (int c = 0; c < l; ++c) bu = fmaf(sB[r * l + c], ub[c * m], bu);
                    }
                    d[q] = xv;
                    d[S::SP + q] = bu;
                }
            };
            // first-layer operand of row r1: [X, BU] of rows r1-1 .. r1+1, hi | lo (warps 4-7)
            const bool f_role = tid >= FM && tid < 2 * FM;
            auto build_f = [&](int r1) {
                const int q = G + (tid - FM);
                __align__(16) __half hi[8], lo[8];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const float* row = xb + mod_pos(r1 - 1 + dy, S::NXB) * 2 * S::SP;
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch) tc::split_f16(row[ch * S::SP + q], hi[2 * dy + ch], lo[2 * dy + ch]);
                }
                hi[6] = hi[7] = lo[6] = lo[7] = __float2half(0.f);
                unsigned char* f = smem + S::OFF_F + (r1 & 1) * S::FBUF + q * 16;
                *reinterpret_cast<uint4*>(f) = *reinterpret_cast<const uint4*>(hi);
                *reinterpret_cast<uint4*>(f + S::PLANE) = *reinterpret_cast<const uint4*>(lo);
            };
            // tanh(main + corr 2^-11 + bias) of this warp's 8 channels -> hi/lo operand row
            auto drain = [&](uint32_t acc, const float* bias, unsigned char* dst) {
                float mv[8], cv[8];
                tmem_ld8(tmem + tlane + acc + cg * 8, mv);
                tmem_ld8(tmem + tlane + acc + C + cg * 8, cv);
                tc::tmem_ld_wait();
                __align__(16) __half hi[8], lo[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tc::split_f16(tanh_fast(fmaf(cv[j], tc::SPLIT_INV, mv[j]) + bias[cg * 8 + j]), hi[j], lo[j]);
                const int q = G + ep;
                *reinterpret_cast<uint4*>(dst + cg * S::PLANE + q * 16) = *reinterpret_cast<const uint4*>(hi);
                *reinterpret_cast<uint4*>(dst + (S::KC + cg) * S::PLANE + q * 16) = *reinterpret_cast<const uint4*>(lo);
            };
            // this warp's operand writes (and TMEM reads) are done: one arrival
            auto arrive = [&](int i) {
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(mb + i);
            };

            for (int r = r_lo - 2; r <= r_lo; ++r) store_xb(r, fetch_x(r));
            float xpf = fetch_x(r_lo + 1);               // next [X; B U] row, in flight
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;          // outputs of rows h-1, h, h+1 (warps 0-3)

            // iteration k: drain first-layer row k+2 and hidden row k, finish the
            // last layer of row k-1 (output row k-2), build first-layer row k+4
            for (int k = r_lo - 5; k <= r_hi + 1; ++k) {
                if (tc::named_bar_or(BAR_DRAIN, ND, failed)) { failed = true; break; }
                tc::fence_after_sync();
                if (Fvalid(k + 2)) {
                    // its slot held row k-2, last read by hidden row k-1 (done)
                    wait(MB_F);
                    drain(S::T_F + ((k + 2) & 1) * 64, sbias, smem + S::OFF_H1 + mod_pos(k + 2, S::NH1) * S::SLOT);
                    arrive(MB_RH1);
                }
                if (k >= r_lo && k <= r_hi) {
                    // its buffer held row k-2, read by last(k-2) (done: waited by
                    // warps 0-3 before the barrier above)
                    wait(MB_H + (k & 1));
                    drain(S::T_H + (k & 1) * 64, sbias + C, smem + S::OFF_H2 + (k & 1) * S::SLOT);
                    arrive(MB_RH2 + (k & 1));
                }
                // last layer of hidden row h = k-1: contributions to output rows h+1, h, h-1
                if (warp < 4 && k - 1 >= r_lo && k - 1 <= r_hi) {
                    wait(MB_L + ((k - 1) & 1));
                    float v[8];
                    tmem_ld8(tmem + tlane + S::T_L + ((k - 1) & 1) * 16, v);
                    tc::tmem_ld_wait();
                    const float p0 = fmaf(v[3], tc::SPLIT_INV, v[0]);
                    const float p1 = fmaf(v[4], tc::SPLIT_INV, v[1]);
                    const float p2 = fmaf(v[5], tc::SPLIT_INV, v[2]);
                    a0 += p2;
                    a1 += p1;
                    a2 += p0;
                    const int ro = k - 2;
                    if (ro >= ys && ro < ye) {
                        const int b = ep % G, x = ep / G, mbr = g * G + b;
                        if (mbr < Nb) {
                            const float xv = xb[mod_pos(ro, S::NXB) * 2 * S::SP + G + ep];
                            Xout[(long)mbr * o_ms + (long)ro * m + x] = fmaf(rs, a0 + sbias[2 * C], xv);
                        }
                    }
                    a0 = a1; a1 = a2; a2 = 0.f;
                }
                // operand of first-layer row k+4 (its buffer held row k+2, whose
                // MMA was waited for above), [X; B U] row k+6
                if (f_role && Fvalid(k + 4)) {
                    build_f(k + 4);
                    arrive(MB_RF + ((k + 4) & 1));
                }
                store_xb(k + 6, xpf);
                xpf = fetch_x(k + 7);
            }
            if (!failed && ye == n && warp < 4) {
                // bottom row: the hidden row below the image is zero
                const int b = ep % G, x = ep / G, mbr = g * G + b;
                if (mbr < Nb) {
                    const float xv = xb[mod_pos(n - 1, S::NXB) * 2 * S::SP + G + ep];
                    Xout[(long)mbr * o_ms + (long)(n - 1) * m + x] = fmaf(rs, a0 + sbias[2 * C], xv);
                }
            }
        }
        tc::fence_before_sync();
        if (__syncthreads_or(failed)) { failed = true; break; }
        tc::fence_after_sync();
    }
    // every MMA issued has landed before the tensor memory is released
    if (warp == ND / 32 && lane == 0) {
        tc::mma_commit(mb + MB_FIN);
        if (!tc::mbar_wait_bounded(mb + MB_FIN, 0u, F_WAIT)) atomicExch(err, DEV_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

template <int C, int G>
size_t fused_smem(int n, int l)
{
    using S = FS<C, G>;
    return (size_t)S::OFF_DYN + sizeof(float) * ((size_t)G * l * (FM / G) + (size_t)n * l) + 16;
}

template <int C, int G>
int fused_launch(const float* X, long x_ms, const float* U, long u_ms, float* Xout, long o_ms,
                 const float* Bmat, int Nb, int n, int l, const float* b1, const void* wpk2, const float* b2,
                 const void* wpk13, const float* b3, float rs, int n_sm, int* err, cudaStream_t st)
{
    const size_t smem = fused_smem<C, G>(n, l);
    if (smem > 227 * 1024) return 1;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(cnn_fused_kernel<C, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024) != cudaSuccess)
            return 1;
        configured = true;
    }
    const long tiles = (long)((Nb + G - 1) / G) * n;
    const int grid = (int)(tiles < n_sm ? tiles : n_sm);
    cnn_fused_kernel<C, G><<<grid, FT, smem, st>>>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1,
                                                  static_cast<const __half*>(wpk2), b2,
                                                  static_cast<const __half*>(wpk13), b3, rs, err);
    return 0;
}

}  // namespace

bool cnn_fused_supported(int n_layers, const int* channels, int n, int m, int l)
{
    if (n_layers != 3 || channels[1] != 32 || channels[2] != 32) return false;
    if (!(m == 16 || m == 32 || m == 64 || m == 128)) return false;
    const int G = FM / m;
    const size_t dyn = sizeof(float) * ((size_t)G * l * m + (size_t)n * l);
    return (size_t)FS<32, 8>::OFF_DYN + dyn + 16 <= 227 * 1024;
}

size_t cnn_fused_packed_bytes() { return (size_t)FS<32, 1>::B1BYTES + FS<32, 1>::B3BYTES; }

// First-layer tiles (3 taps): [kc][64 rows][8]; rows 0..31 main = [w_hi(6), 0, 0 | 0],
// rows 32..63 corr = [w_lo(6), 0, 0 | w_hi(6), 0, 0], with K index e = 2 dy + ch.
// Last-layer tiles (3 taps x 2 K-steps x {B1, B2}): [kc][16 rows][8]; B1 rows
// 0..2 = w_hi of stencil rows 0..2, rows 3..5 = w_lo; B2 rows 3..5 = w_hi.
void cnn_fused_pack_weights(const float* w1, const float* w3, void* dst_host)
{
    constexpr int C = 32;
    __half* out = static_cast<__half*>(dst_host);
    const size_t n1 = FS<C, 1>::B1BYTES / 2, n3 = FS<C, 1>::B3BYTES / 2;
    for (size_t i = 0; i < n1 + n3; ++i) out[i] = __float2half(0.f);
    auto split = [](float v, __half& hi, __half& lo) {
        hi = __float2half_rn(v);
        lo = __float2half_rn((v - __half2float(hi)) * tc::SPLIT_SCALE);
    };
    for (int dx = 0; dx < 3; ++dx)
        for (int co = 0; co < C; ++co)
            for (int e = 0; e < 6; ++e) {
                const int dy = e / 2, ch = e % 2;
                __half hi, lo;
                split(w1[((co * 2 + ch) * 3 + dy) * 3 + dx], hi, lo);
                __half* t = out + (size_t)dx * 2 * 64 * 8;
                t[(0 * 64 + co) * 8 + e] = hi;              // main: kc 0
                t[(0 * 64 + 32 + co) * 8 + e] = lo;         // corr: kc 0 lo
                t[(1 * 64 + 32 + co) * 8 + e] = hi;         // corr: kc 1 hi
            }
    __half* l3 = out + n1;
    for (int dx = 0; dx < 3; ++dx)
        for (int ks = 0; ks < C / 16; ++ks)
            for (int kc = 0; kc < 2; ++kc)
                for (int e = 0; e < 8; ++e) {
                    const int ci = ks * 16 + kc * 8 + e;
                    for (int d = 0; d < 3; ++d) {
                        __half hi, lo;
                        split(w3[(ci * 3 + d) * 3 + dx], hi, lo);
                        __half* b1 = l3 + (size_t)((dx * (C / 16) + ks) * 2 + 0) * (2 * 16 * 8);
                        __half* b2 = l3 + (size_t)((dx * (C / 16) + ks) * 2 + 1) * (2 * 16 * 8);
                        b1[(kc * 16 + d) * 8 + e] = hi;
                        b1[(kc * 16 + 3 + d) * 8 + e] = lo;
                        b2[(kc * 16 + 3 + d) * 8 + e] = hi;
                    }
                }
}

int launch_cnn_fused(const float* X, long x_ms, const float* U, long u_ms, float* Xout, long o_ms,
                     const float* Bmat, int Nb, int n, int m, int l, const float* b1, const void* wpk2,
                     const float* b2, const void* wpk13, const float* b3, float rs, int n_sm, int* err,
                     cudaStream_t st)
{
    switch (m) {
    case 128: return fused_launch<32, 1>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, wpk2, b2, wpk13, b3, rs, n_sm, err, st);
    case 64: return fused_launch<32, 2>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, wpk2, b2, wpk13, b3, rs, n_sm, err, st);
    case 32: return fused_launch<32, 4>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, wpk2, b2, wpk13, b3, rs, n_sm, err, st);
    case 16: return fused_launch<32, 8>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, wpk2, b2, wpk13, b3, rs, n_sm, err, st);
    }
    return 1;
}

}  // namespace oic
