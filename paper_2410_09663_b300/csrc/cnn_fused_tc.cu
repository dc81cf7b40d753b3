// cnn_fused_tc.cu -- the whole surrogate X_{t+1} = X_t + s * CNN_theta(X_t, U_t)
// of Eq. (1), structure [X; B U] -> C (tanh) -> C (tanh) -> 1, in ONE kernel,
// every layer on the tcgen05 tensor cores at FP32 accuracy.
//
// Precision: operands are split x = hi + lo * 2^-11 (hi, lo fp16) and each
// layer accumulates main = A_hi B_hi and corr = A_hi B_lo + A_lo B_hi in
// tensor memory (out = main + corr * 2^-11, error ~2^-21 per product).
//
// Layout: a CTA owns a group of G = 128/m members; an M = 128 tile is one
// image row of the group with the members INTERLEAVED pixel by pixel
// (position G + G x + b for member b, pixel x, zero pads at both ends), so a
// horizontal stencil tap is a shift of the operand start by G positions.
//
// One MMA costs at least ~50 cycles whatever its N up to 64, and runs at the
// full tensor rate only from N = 128 up, so each layer is cast into few wide
// MMAs:
//   first layer (2 -> C)   K = 16 per horizontal tap holds [X, B U] of the
//                          three stencil rows, hi and lo; N = 2C (main, corr)
//   hidden layer (C -> C)  the three VERTICAL taps are stacked along N: one
//                          first-layer row j, read once per (horizontal tap,
//                          16-channel step), feeds hidden rows j+1, j, j-1 at
//                          once (N = 6C).  Hidden-row accumulators live in a
//                          ring of 4 TMEM slots whose window of three is
//                          contiguous except at the ring's end (then split)
//   last layer (C -> 1)    all nine taps are stacked along N (main and corr
//                          of each, N = 32) on the UNshifted row; the CUDA
//                          cores add the horizontal neighbours (+-G lanes,
//                          through shared memory) and keep rolling sums over
//                          output rows h+1, h, h-1
//
// Roles: one warp (20) issues the MMAs (an elected lane each, operands warp-
// uniform) and waits only on "operand ready" /
// "accumulator drained" mbarriers; 16 drain warps turn accumulators into the
// next layer's operands (tanh, split, stores), four of them (2, 3, 6, 7) also
// building the first layer's operand rows; 4 warps (16-19) finish the last
// layer (neighbour sums, residual, X_next), warp 17 issuing its MMAs.  Both
// wait on the MMA commit barriers.
// Only X, U and the weights are read and X_next written (X_next must not
// overlap X: neighbouring CTAs read halo rows of X).  The grid is persistent
// over contiguous (group, row) ranges.
#include <cuda_fp16.h>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int FT = 672;                                 // 16 drain + 4 last-layer + 1 MMA-issuing warp
constexpr int ND = 512;                                 // drain threads (warps 0-15)
constexpr int FM = 128;                                 // tile rows (pixels)
constexpr int BAR_DRAIN = 1;                            // named barrier of the drain warps (segment start)
constexpr int BAR_E3 = 2;                               // named barrier of the last-layer warps
constexpr int E3_WARP0 = 16;                            // warps 16-19 finish the last layer
constexpr int E3_ISSUE = E3_WARP0 + 1;                  // the one of them that issues its MMAs (warp 17:
                                                        // not on the main issuing warp's scheduler)
constexpr int ISSUE_WARP = 20;
constexpr long long F_WAIT = 4000000000LL;

__host__ __device__ constexpr int al16(int x) { return (x + 15) / 16 * 16; }

template <int C, int G>
struct FS {
    static constexpr int KC = C / 8, KS = C / 16;
    static constexpr int NPOS = FM + 2 * G;             // operand positions incl. pads
    static constexpr int PLANE = NPOS * 16;             // one (part, 8-channel) plane
    static constexpr int SLOT = 2 * KC * PLANE;         // hi and lo of one activation row
    static constexpr int FBUF = 2 * PLANE;              // first-layer operand: hi | lo
    static constexpr int HROWS = 6 * C;                 // hidden B tile rows: 3 x [B_hi; B_lo]
    static constexpr int HTILE = 2 * HROWS * 16;        // one (tap, K-step, part) tile, 2 K chunks
    static constexpr int BBYTES = 3 * KS * 2 * HTILE;   // [dx][ks][hi | lo]
    static constexpr int B1BYTES = 3 * 2 * 64 * 16;     // first layer: 3 taps x (2 x 64 x 8)
    static constexpr int B3TILE = 2 * 32 * 16;          // last layer tile: 2 K chunks x 32 rows
    static constexpr int B3BYTES = KS * 2 * B3TILE;     // [ks][hi | lo]
    static constexpr int OFF_H1 = 0;                    // first-layer rows, 2 slots
    static constexpr int OFF_H2 = OFF_H1 + 2 * SLOT;    // hidden rows, 2 slots
    static constexpr int OFF_F = OFF_H2 + 2 * SLOT;     // first-layer operands, 2 buffers
    static constexpr int OFF_EX = OFF_F + 2 * FBUF;     // last-layer neighbour exchange [2][6][NPOS] fp32
    static constexpr int EXBYTES = al16(2 * 6 * NPOS * 4);
    static constexpr int ZERO_BYTES = OFF_EX + EXBYTES; // operand buffers incl. pads
    static constexpr int OFF_B = ZERO_BYTES;
    static constexpr int OFF_B1 = OFF_B + BBYTES;
    static constexpr int OFF_B3 = OFF_B1 + B1BYTES;
    static constexpr int PACKED = BBYTES + B1BYTES + B3BYTES;
    static constexpr int OFF_BIAS = OFF_B3 + B3BYTES;                  // b1[C], b2[C], b3
    static constexpr int OFF_MISC = OFF_BIAS + al16((2 * C + 4) * 4);  // mbarriers, TMEM base
    static constexpr int OFF_DYN = OFF_MISC + 128;                     // U group, B matrix
    // tensor memory: hidden ring (4 x [main | corr]), first layer (2 x [main | corr]),
    // last layer (2 x 32)
    static constexpr int T_H = 0, T_F = 8 * C, T_L = 12 * C;
    static constexpr int TMEM_COLS = 512;
    static_assert(T_L + 64 <= TMEM_COLS, "tensor memory");
};

// tanh(x) = 1 - 2 / (1 + e^{2x}): saturates correctly at both ends; absolute
// error a few 1e-7 (the exponential and the quotient are each within a few
// ulps), which is below the FP32 rounding of the layer's inputs.
__device__ __forceinline__ float tanh_fast(float x)
{
    return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x));
}

// Two values split at once: hi = fp16 rounding of (y0, y1), lo = fp16 of the
// residuals scaled by 2^11 (packed conversions).
__device__ __forceinline__ void split2(float y0, float y1, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(y0, y1);
    const float2 b = __half22float2(h);
    const __half2 l = __floats2half2_rn((y0 - b.x) * tc::SPLIT_SCALE, (y1 - b.y) * tc::SPLIT_SCALE);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
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

// Shared-memory operand descriptors are handled as their low 32-bit word
// (address >> 4 in bits [0,14), leading byte offset >> 4 in bits [16,30));
// the high word is the same for every operand here (stride byte offset 128,
// descriptor version 1).  Every shared address is below 256 KB, so adding a
// byte offset >> 4 to the low word never carries out of the address field.
constexpr uint32_t DESC_HI = (128u >> 4) | (1u << 14);
__host__ __device__ constexpr uint32_t desc_lo(uint32_t saddr, uint32_t lbo)
{
    return ((saddr & 0x3FFFFu) >> 4) | (((lbo >> 4) & 0x3FFFu) << 16);
}

// One MMA from descriptor low words (see tc::mma_f16), called by a whole
// warp with warp-uniform operands: the elected lane issues it.  Keeping the
// issue loop warp-wide lets the operands stay in uniform registers; issued
// from one lane's divergent branch, each MMA paid for moving them there
// (measured: the MMA issue of a row pass 2.45k -> 1.72k cycles, the CNN step
// 124.7 -> 118.5 us at 64 x 64, N = 256).
__device__ __forceinline__ void mma_lo(uint32_t d_tmem, uint32_t a_lo, uint32_t b_lo, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .b64 da, db;\n\t.reg .pred p, e;\n\t"
        "mov.b64 da, {%1, %5};\n\t"
        "mov.b64 db, {%2, %5};\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_lo), "r"(b_lo), "r"(idesc), "r"(acc), "r"(DESC_HI)
        : "memory");
}

// First layer of row r1: a = descriptor of its operand buffer, b = of the tiles.
template <int C, int G>
__device__ __forceinline__ void issue_first(uint32_t acc, uint32_t a, uint32_t b)
{
    constexpr uint32_t id = tc::idesc_f16(FM, 64);
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) mma_lo(acc, a + dx * G, b + dx * (2048 >> 4), id, dx > 0 ? 1u : 0u);
}

// MMA over the vertical-tap blocks [B0, B1) of one hidden B tile into TMEM
// from column COL (blocks are 2C columns wide: main | corr).  The lo part
// writes only the corr halves: N = 2C (B1 - B0) - C from column COL + C.
template <int C, int B0, int B1, int COL, bool LO>
__device__ __forceinline__ void hid_piece(uint32_t tmem, uint32_t a, uint32_t b, uint32_t acc)
{
    constexpr int NN = LO ? 2 * C * (B1 - B0) - C : 2 * C * (B1 - B0);
    constexpr uint32_t id = tc::idesc_f16(FM, NN);
    constexpr uint32_t brow = 2 * C * B0 + (LO ? C : 0);
    mma_lo(tmem + COL + (LO ? C : 0), a, b + brow, id, acc);
}

// All hidden-layer MMAs of first-layer row j.  Blocks b = 0, 1, 2 hold
// vertical taps dy = b, i.e. hidden rows j+1, j, j-1, whose ring slots are
// SR, SR+1, SR+2 (mod 4) with SR = (-j-1) mod 4.  The first MMA starts hidden
// row j+1 (accumulate = 0 on its block); with INIT_ALL it starts every block.
// a = descriptor of the row's operand slot, b = of the hidden tiles.
template <int C, int G, int SR, bool INIT_ALL>
__device__ __forceinline__ void issue_hidden_s(uint32_t tmem, uint32_t a, uint32_t b)
{
    using S = FS<C, G>;
    constexpr int W = 2 * C;                            // ring slot width in columns
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
        for (int ks = 0; ks < S::KS; ++ks) {
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const uint32_t aa = a + (((part ? S::KC : 0) + 2 * ks) * S::PLANE) / 16 + dx * G;
                const uint32_t bb = b + (((dx * S::KS + ks) * 2 + part) * S::HTILE) / 16;
                const bool first = dx == 0 && ks == 0 && part == 0;
                if (part == 0) {
                    if (first && !INIT_ALL) {
                        // block 0 alone with accumulate = 0, blocks 1-2 accumulate
                        hid_piece<C, 0, 1, S::T_H + W * SR, false>(tmem, aa, bb, 0u);
                        if constexpr (SR == 2) {
                            hid_piece<C, 1, 2, S::T_H + W * 3, false>(tmem, aa, bb, 1u);
                            hid_piece<C, 2, 3, S::T_H, false>(tmem, aa, bb, 1u);
                        } else if constexpr (SR == 3) {
                            hid_piece<C, 1, 3, S::T_H, false>(tmem, aa, bb, 1u);
                        } else {
                            hid_piece<C, 1, 3, S::T_H + W * (SR + 1), false>(tmem, aa, bb, 1u);
                        }
                        continue;
                    }
                }
                const uint32_t acc = first ? 0u : 1u;
                if (part == 0) {
                    if constexpr (SR <= 1) {
                        hid_piece<C, 0, 3, S::T_H + W * SR, false>(tmem, aa, bb, acc);
                    } else if constexpr (SR == 2) {
                        hid_piece<C, 0, 2, S::T_H + W * 2, false>(tmem, aa, bb, acc);
                        hid_piece<C, 2, 3, S::T_H, false>(tmem, aa, bb, acc);
                    } else {
                        hid_piece<C, 0, 1, S::T_H + W * 3, false>(tmem, aa, bb, acc);
                        hid_piece<C, 1, 3, S::T_H, false>(tmem, aa, bb, acc);
                    }
                } else {
                    if constexpr (SR <= 1) {
                        hid_piece<C, 0, 3, S::T_H + W * SR, true>(tmem, aa, bb, 1u);
                    } else if constexpr (SR == 2) {
                        hid_piece<C, 0, 2, S::T_H + W * 2, true>(tmem, aa, bb, 1u);
                        hid_piece<C, 2, 3, S::T_H, true>(tmem, aa, bb, 1u);
                    } else {
                        hid_piece<C, 0, 1, S::T_H + W * 3, true>(tmem, aa, bb, 1u);
                        hid_piece<C, 1, 3, S::T_H, true>(tmem, aa, bb, 1u);
                    }
                }
            }
        }
    }
}

// Dispatch on the ring position once per row, so that the MMA sequence itself
// is straight-line code.
template <int C, int G>
__device__ __forceinline__ void issue_hidden(uint32_t tmem, int j, bool init_all, uint32_t a, uint32_t b)
{
    const int s = (-j - 1) & 3;
    if (init_all) {
        switch (s) {
        case 0: issue_hidden_s<C, G, 0, true>(tmem, a, b); break;
        case 1: issue_hidden_s<C, G, 1, true>(tmem, a, b); break;
        case 2: issue_hidden_s<C, G, 2, true>(tmem, a, b); break;
        default: issue_hidden_s<C, G, 3, true>(tmem, a, b); break;
        }
    } else {
        switch (s) {
        case 0: issue_hidden_s<C, G, 0, false>(tmem, a, b); break;
        case 1: issue_hidden_s<C, G, 1, false>(tmem, a, b); break;
        case 2: issue_hidden_s<C, G, 2, false>(tmem, a, b); break;
        default: issue_hidden_s<C, G, 3, false>(tmem, a, b); break;
        }
    }
}

// Last layer of hidden row h, all nine taps along N, on the unshifted row:
// a = descriptor of the row's operand buffer (centre tap), b = of the tiles.
template <int C, int G>
__device__ __forceinline__ void issue_last(uint32_t acc, uint32_t a, uint32_t b)
{
    using S = FS<C, G>;
    constexpr uint32_t id = tc::idesc_f16(FM, 32);
#pragma unroll
    for (int ks = 0; ks < S::KS; ++ks) {
#pragma unroll
        for (int part = 0; part < 2; ++part)
            mma_lo(acc, a + (((part ? S::KC : 0) + 2 * ks) * S::PLANE) / 16, b + ((ks * 2 + part) * S::B3TILE) / 16,
                   id, (ks | part) ? 1u : 0u);
    }
}

// mbarriers in the MISC region (8 bytes each); [2] = by row parity
enum : int {
    MB_F = 0,          // [2] first layer of row f done (tensor core -> drain warps)
    MB_H = 2,          // [2] hidden MMAs of first-layer row j done
    MB_L = 4,          // [2] last layer of hidden row h done
    MB_W1 = 6,         // [2] drain pass k-1 done: first-layer row k in its slot, operand
                       //     of first-layer row k+2 built (16 drain warps)
    MB_W2 = 8,         // [2] hidden row h in its buffer (16 drain warps)
    MB_FIN = 10,       // every MMA of the kernel done
    MB_COUNT = 11
};

// Ordering used below: tcgen05.commit signals completion of ALL earlier MMAs
// of the committing thread.  The first- and hidden-layer MMAs come from one
// thread (the issuing warp's elected lane: lane 0, the warp being converged)
// in the order first(k+2), hidden(k), so the wait for hidden(k) also covers
// first(k+1).  The last-layer MMAs come from the elected lane of the first
// last-layer warp, which issues last(h) once hidden row h is in its buffer.
template <int C, int G>
__global__ void __launch_bounds__(FT, 1)
cnn_fused_kernel(const float* __restrict__ X, long x_ms, const float* __restrict__ U, long u_ms,
                 float* __restrict__ Xout, long o_ms, const float* __restrict__ Bmat, int Nb, int n, int l,
                 const float* __restrict__ b1, const float* __restrict__ b2, const float* __restrict__ b3,
                 const __half* __restrict__ wpk, float rs, int* __restrict__ err, UAdvance ua)
{
    pdl_trigger();
    using S = FS<C, G>;
    static_assert(C == 32, "16 drain warps = 4 lane quarters x 4 groups of 8 channels");
    static_assert(MB_COUNT * 8 + 4 <= 128, "MISC region");
    static_assert(FT == 32 * (ISSUE_WARP + 1) && E3_WARP0 * 32 == ND, "warp roles");
    constexpr int m = FM / G;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* ex = reinterpret_cast<float*>(smem + S::OFF_EX);
    float* sbias = reinterpret_cast<float*>(smem + S::OFF_BIAS);   // b1 | b2 | b3
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + S::OFF_MISC);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::OFF_MISC + MB_COUNT * 8);
    float* su = reinterpret_cast<float*>(smem + S::OFF_DYN);                 // [G][m][l]
    float* sB = su + G * l * m;                                              // [n][l]
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t s0 = tc::smem_u32(smem);

    // ---- one-time set-up: zero the operand buffers (pads stay zero), copy weights
    for (int e = tid; e < S::ZERO_BYTES / 16; e += FT)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < S::PACKED / 16; e += FT)
        reinterpret_cast<uint4*>(smem + S::OFF_B)[e] = reinterpret_cast<const uint4*>(wpk)[e];
    for (int e = tid; e < C; e += FT) { sbias[e] = b1[e]; sbias[C + e] = b2[e]; }
    for (int e = tid; e < n * l; e += FT) sB[e] = Bmat[e];
    if (tid == 0) {
        sbias[2 * C] = b3[0];
        for (int i = 0; i < MB_COUNT; ++i) {
            const int cnt = (i >= MB_W1 && i < MB_W2 + 2) ? 16 : 1;
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
    pdl_wait();                                         // the set-up above reads no kernel's output

    const int groups = (Nb + G - 1) / G;
    const long total = (long)groups * n;
    const long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    uint32_t ph = 0;                                    // this thread's phase bit per mbarrier
    bool failed = false;
    auto wait = [&](int i) {
        if (!tc::mbar_wait_backoff(mb + i, (ph >> i) & 1u, F_WAIT)) {
            failed = true;
            atomicExch(err, DEV_TIMEOUT);
        }
        ph ^= 1u << i;
        tc::fence_after_sync();
    };
    // the same by all 32 lanes of a warp, which then agree on the outcome
    // (every later warp-wide step is taken by all lanes or by none)
    auto wait_w = [&](int i) {
        wait(i);
        failed = __any_sync(0xffffffffu, failed);
    };
    // a phase this thread knows to be complete without waiting for it
    auto passed = [&](int i) { ph ^= 1u << i; };
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
        // rows f_lo .. f_hi (zero outside the image)
        const int r_lo = ys > 0 ? ys - 1 : 0;
        const int r_hi = ye < n ? ye : n - 1;
        const int f_lo = r_lo - 1 > 0 ? r_lo - 1 : 0;
        const int f_hi = r_hi + 1 < n - 1 ? r_hi + 1 : n - 1;
        auto Fv = [&](int f) { return f >= f_lo && f <= f_hi; };
        auto Hv = [&](int h) { return h >= r_lo && h <= r_hi; };

        if (warp == ISSUE_WARP) {
            // ================= MMA-issuing warp (elected lane) =================
            {
                const uint32_t dH1 = desc_lo(s0 + S::OFF_H1, S::PLANE);           // first-layer rows (A)
                const uint32_t dHB = desc_lo(s0 + S::OFF_B, S::HROWS * 16);       // hidden tiles (B)
                const uint32_t dF = desc_lo(s0 + S::OFF_F, S::PLANE);             // first-layer operands (A)
                const uint32_t dB1 = desc_lo(s0 + S::OFF_B1, 64 * 16);            // first-layer tiles (B)
                for (int k = f_lo - 2; k <= r_hi + 1 && !failed; ++k) {
                    wait_w(MB_W1 + (k & 1));                        // drain pass k-1
                    if (Fv(k + 2)) {
                        issue_first<C, G>(tmem + S::T_F + ((k + 2) & 1) * 2 * C,
                                          dF + ((k + 2) & 1) * (S::FBUF / 16), dB1);
                        tc::mma_commit_elect(mb + MB_F + ((k + 2) & 1));
                    }
                    if (Fv(k)) {
                        issue_hidden<C, G>(tmem, k, k == f_lo, dH1 + (k & 1) * (S::SLOT / 16), dHB);
                        tc::mma_commit_elect(mb + MB_H + (k & 1));
                    }
                }
            }
            __syncwarp();
        } else if (warp >= E3_WARP0) {
            // ================= 4 last-layer warps =================
            // hidden row h: its nine tap products at every pixel -> contributions
            // to output rows h+1, h, h-1; output row h-1 is then complete
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;          // outputs of rows h-1, h, h+1
            const int b = ep % G, x = ep / G, mbr = g * G + b;
            const uint32_t dH2 = desc_lo(s0 + S::OFF_H2 + G * 16, S::PLANE);      // hidden rows, centre (A)
            const uint32_t dB3 = desc_lo(s0 + S::OFF_B3, 32 * 16);                // last-layer tiles (B)
            for (int h = r_lo; h <= r_hi; ++h) {
                if (warp == E3_ISSUE) {
                    // hidden row h in its buffer; its accumulator buffer was read
                    // out for row h-2 by all four warps before the last barrier
                    wait_w(MB_W2 + (h & 1));
                    issue_last<C, G>(tmem + S::T_L + (h & 1) * 32, dH2 + (h & 1) * (S::SLOT / 16), dB3);
                    tc::mma_commit_elect(mb + MB_L + (h & 1));
                }
                wait_w(MB_L + (h & 1));
                float v[8], w[8], z[8];
                const uint32_t ta = tmem + tlane + S::T_L + (h & 1) * 32;
                tmem_ld8(ta, v);          // main of taps 0-7
                tmem_ld8(ta + 8, w);      // main of tap 8, corr of taps 0-6
                tmem_ld8(ta + 16, z);     // corr of taps 7-8
                tc::tmem_ld_wait();
                tc::fence_before_sync();
                // tap t = 3 dy + dx: main in column t, corr in column 9 + t
                float P[9];
#pragma unroll
                for (int tp = 0; tp < 9; ++tp) {
                    const float mn = tp < 8 ? v[tp] : w[0];
                    const float cr = tp < 7 ? w[1 + tp] : z[tp - 7];
                    P[tp] = fmaf(cr, tc::SPLIT_INV, mn);
                }
                // horizontal neighbours: output pixel x takes tap dx from
                // hidden pixel x + dx - 1, i.e. lane ep + (dx - 1) G
                float* e0 = ex + (h & 1) * 6 * S::NPOS;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    e0[(2 * dy) * S::NPOS + G + ep] = P[3 * dy];
                    e0[(2 * dy + 1) * S::NPOS + G + ep] = P[3 * dy + 2];
                }
                if (tc::named_bar_or(BAR_E3, 4 * 32, failed)) { failed = true; break; }
                tc::fence_after_sync();
                float c3[3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
                    c3[dy] = P[3 * dy + 1] + e0[(2 * dy) * S::NPOS + ep] + e0[(2 * dy + 1) * S::NPOS + 2 * G + ep];
                a0 += c3[2];
                a1 += c3[1];
                a2 += c3[0];
                const int ro = h - 1;
                if (ro >= ys && ro < ye && mbr < Nb)
                    Xout[(long)mbr * o_ms + (long)ro * m + x] =
                        fmaf(rs, a0 + sbias[2 * C], X[(long)mbr * x_ms + (long)ro * m + x]);
                a0 = a1; a1 = a2; a2 = 0.f;
            }
            if (!failed && ye == n && mbr < Nb) {
                // bottom row: the hidden row below the image is zero
                Xout[(long)mbr * o_ms + (long)(n - 1) * m + x] =
                    fmaf(rs, a0 + sbias[2 * C], X[(long)mbr * x_ms + (long)(n - 1) * m + x]);
            }
        } else {
            // ================= 16 drain warps =================
            // U of the group, transposed to [member][pixel][control] so that one
            // pixel's l controls are contiguous
            // (the segment that starts at row 0 also advances U_t = U_{t-1} + W)
            const bool adv = ua.next != nullptr && ys == 0;
            for (int e = tid; e < G * l * m; e += ND) {
                const int b = e / (l * m), rr = e % (l * m), c = rr / m, xx = rr % m;
                const int mbr = g * G + b;
                const float uv = mbr < Nb ? U[(long)mbr * u_ms + rr] : 0.f;
                su[(b * m + xx) * l + c] = uv;
                if (adv && mbr < Nb) ua.next[(long)mbr * u_ms + rr] = uv + noise1(ua.w, (long)mbr * l * m + rr);
            }
            tc::named_bar(BAR_DRAIN, ND);

            // four drain warps build the first-layer operands: thread p owns position
            // G + p (member p % G, pixel p / G) and keeps [X, B U] of the three
            // rows it needs in registers
            // (drain warps 2, 3, 6 and 7: on schedulers 2 and 3, away from the two
            // MMA-issuing warps on schedulers 0 and 1)
            const bool f_role = (warp & 2) != 0 && warp < 8;
            const int fp = f_role ? tid - (warp < 4 ? 64 : 128) : 0;
            const int f_b = fp % G, f_x = fp / G, f_mb = g * G + f_b;
            auto fetch_x = [&](int r) -> float {
                return (f_role && r >= 0 && r < n && f_mb < Nb) ? X[(long)f_mb * x_ms + (long)r * m + f_x] : 0.f;
            };
            auto bu_of = [&](int r) -> float {
                float bu = 0.f;
                if (f_role && r >= 0 && r < n && f_mb < Nb) {
                    const float* ub = su + (f_b * m + f_x) * l;
                    const float* bb = sB + r * l;
                    if ((l & 3) == 0) {
                        for (int c = 0; c < l; c += 4) {
                            const float4 u4 = *reinterpret_cast<const float4*>(ub + c);
                            const float4 b4 = *reinterpret_cast<const float4*>(bb + c);
                            bu = fmaf(b4.x, u4.x, fmaf(b4.y, u4.y, fmaf(b4.z, u4.z, fmaf(b4.w, u4.w, bu))));
                        }
                    } else {
                        for (int c = 0; c < l; ++c) bu = fmaf(bb[c], ub[c], bu);
                    }
                }
                return bu;
            };
            float xr[3], br[3];                           // rows k+2 .. k+4 at pass k
#pragma unroll
            for (int i = 0; i < 3; ++i) { xr[i] = fetch_x(f_lo - 1 + i); br[i] = bu_of(f_lo - 1 + i); }
            float xpf = fetch_x(f_lo + 2);                // row k+5, in flight
            auto build_f = [&](int r1) {
                uint32_t hi[3], lo[3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) split2(xr[dy], br[dy], hi[dy], lo[dy]);
                unsigned char* f = smem + S::OFF_F + (r1 & 1) * S::FBUF + (G + fp) * 16;
                *reinterpret_cast<uint4*>(f) = make_uint4(hi[0], hi[1], hi[2], 0u);
                *reinterpret_cast<uint4*>(f + S::PLANE) = make_uint4(lo[0], lo[1], lo[2], 0u);
            };
            // tanh(main + corr 2^-11 + bias) of this warp's 8 channels -> hi/lo operand row
            auto drain = [&](uint32_t acc, const float* bias, unsigned char* dst) {
                float mv[8], cv[8];
                tmem_ld8(tmem + tlane + acc + cg * 8, mv);
                tmem_ld8(tmem + tlane + acc + C + cg * 8, cv);
                tc::tmem_ld_wait();
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float y0 = tanh_fast(fmaf(cv[2 * j], tc::SPLIT_INV, mv[2 * j]) + bias[cg * 8 + 2 * j]);
                    const float y1 = tanh_fast(fmaf(cv[2 * j + 1], tc::SPLIT_INV, mv[2 * j + 1]) + bias[cg * 8 + 2 * j + 1]);
                    split2(y0, y1, hi[j], lo[j]);
                }
                const int q = G + ep;
                *reinterpret_cast<uint4*>(dst + cg * S::PLANE + q * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(dst + (S::KC + cg) * S::PLANE + q * 16) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            };
            // this warp's operand writes (and TMEM reads) are done: one arrival
            auto arrive = [&](int i) {
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(mb + i);
            };

            // pass k: drain first-layer row k+1, build the operand of first-layer
            // row k+3, then drain hidden row k-1
            for (int k = f_lo - 3; k <= r_hi + 2 && !failed; ++k) {
                if (Fv(k + 1)) {
                    // first(k+1) precedes hidden(k-1), waited for in pass k-1
                    if (Fv(k - 1)) passed(MB_F + ((k + 1) & 1));
                    else wait_w(MB_F + ((k + 1) & 1));
                    // the slot held first-layer row k-1 (hidden(k-1) done)
                    drain(S::T_F + ((k + 1) & 1) * 2 * C, sbias, smem + S::OFF_H1 + ((k + 1) & 1) * S::SLOT);
                }
                // its buffer held row k+1, read by first(k+1) (done, see above)
                if (f_role && Fv(k + 3)) build_f(k + 3);
                if (k <= r_hi) arrive(MB_W1 + ((k + 1) & 1));   // consumed by issue pass k+1
                if (f_role) {
                    xr[0] = xr[1]; xr[1] = xr[2]; xr[2] = xpf;
                    br[0] = br[1]; br[1] = br[2]; br[2] = bu_of(k + 5);
                    xpf = fetch_x(k + 6);
                }
                if (Fv(k)) wait_w(MB_H + (k & 1));               // hidden MMAs of first-layer row k
                if (Hv(k - 1)) {
                    // hidden row k-1 is complete; its buffer held row k-3, read by
                    // last(k-3)
                    if (Hv(k - 3)) wait_w(MB_L + ((k - 3) & 1));
                    drain(S::T_H + ((-(k - 1)) & 3) * 2 * C, sbias + C, smem + S::OFF_H2 + ((k - 1) & 1) * S::SLOT);
                    arrive(MB_W2 + ((k - 1) & 1));
                }
            }
            // phases of the last two rows' last-layer MMAs (waited for by the
            // last-layer warps before the barrier below)
            // (the drain warps wait for last(h) only when reusing its buffer)
            for (int h = r_hi - 1; h <= r_hi; ++h)
                if (Hv(h)) passed(MB_L + (h & 1));
        }
        tc::fence_before_sync();
        if (__syncthreads_or(failed)) { failed = true; break; }
        tc::fence_after_sync();
    }
    // every MMA issued has landed before the tensor memory is released
    if (warp == ISSUE_WARP && lane == 0) {
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
                 const float* Bmat, int Nb, int n, int l, const float* b1, const float* b2, const float* b3,
                 const void* wpk, float rs, int n_sm, int* err, cudaStream_t st, UAdvance ua)
{
    const size_t smem = fused_smem<C, G>(n, l);
    if (smem > 227 * 1024) return 1;
    static DeviceOnce configured;
    if (!configured.run([] {
            return cudaFuncSetAttribute(cnn_fused_kernel<C, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        227 * 1024) == cudaSuccess;
        }))
        return 1;
    const long tiles = (long)((Nb + G - 1) / G) * n;
    const int grid = (int)(tiles < n_sm ? tiles : n_sm);
    pdl_launch(cnn_fused_kernel<C, G>, grid, FT, smem, st, X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, b2, b3,
                                                  static_cast<const __half*>(wpk), rs, err, ua);
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

size_t cnn_fused_packed_bytes() { return (size_t)FS<32, 1>::PACKED; }

// Packed operand tiles, K-major (8-element core rows of 16 bytes), each
// weight split w = hi + lo 2^-11:
//   hidden [dx][ks][part] tiles of 2 K chunks x 6C rows; row 2C dy + r:
//     part hi: r < C -> w_hi(co = r), else w_lo(co = r - C); part lo: r < C
//     -> 0, else w_hi(co = r - C)
//   first layer [dx] tiles of 2 K chunks x 64 rows; rows 0..31 main =
//     [w_hi(6), 0, 0 | 0], rows 32..63 corr = [w_lo(6), 0, 0 | w_hi(6), 0, 0]
//     with K index e = 2 dy + ch
//   last layer [ks][part] tiles of 2 K chunks x 32 rows; tap t = 3 dy + dx:
//     part hi: row t -> w_hi, row 9 + t -> w_lo; part lo: row 9 + t -> w_hi
void cnn_fused_pack_weights(const float* w1, const float* w2, const float* w3, void* dst_host)
{
    constexpr int C = 32, KS = C / 16;
    using S = FS<C, 1>;
    __half* out = static_cast<__half*>(dst_host);
    for (size_t i = 0; i < (size_t)S::PACKED / 2; ++i) out[i] = __float2half(0.f);
    auto split = [](float v, __half& hi, __half& lo) {
        hi = __float2half_rn(v);
        lo = __float2half_rn((v - __half2float(hi)) * tc::SPLIT_SCALE);
    };
    // hidden
    for (int dx = 0; dx < 3; ++dx)
        for (int ks = 0; ks < KS; ++ks)
            for (int kc = 0; kc < 2; ++kc)
                for (int dy = 0; dy < 3; ++dy)
                    for (int co = 0; co < C; ++co)
                        for (int e = 0; e < 8; ++e) {
                            const int ci = ks * 16 + kc * 8 + e;
                            __half hi, lo;
                            split(w2[((co * C + ci) * 3 + dy) * 3 + dx], hi, lo);
                            __half* th = out + (size_t)((dx * KS + ks) * 2 + 0) * (S::HTILE / 2);
                            __half* tl = out + (size_t)((dx * KS + ks) * 2 + 1) * (S::HTILE / 2);
                            const int r_main = 2 * C * dy + co, r_corr = 2 * C * dy + C + co;
                            th[((size_t)kc * S::HROWS + r_main) * 8 + e] = hi;
                            th[((size_t)kc * S::HROWS + r_corr) * 8 + e] = lo;
                            tl[((size_t)kc * S::HROWS + r_corr) * 8 + e] = hi;
                        }
    // first layer
    __half* f1 = out + S::BBYTES / 2;
    for (int dx = 0; dx < 3; ++dx)
        for (int co = 0; co < C; ++co)
            for (int e = 0; e < 6; ++e) {
                const int dy = e / 2, ch = e % 2;
                __half hi, lo;
                split(w1[((co * 2 + ch) * 3 + dy) * 3 + dx], hi, lo);
                __half* t = f1 + (size_t)dx * 2 * 64 * 8;
                t[(0 * 64 + co) * 8 + e] = hi;              // main: kc 0
                t[(0 * 64 + 32 + co) * 8 + e] = lo;         // corr: kc 0 lo
                t[(1 * 64 + 32 + co) * 8 + e] = hi;         // corr: kc 1 hi
            }
    // last layer
    __half* l3 = f1 + S::B1BYTES / 2;
    for (int ks = 0; ks < KS; ++ks)
        for (int kc = 0; kc < 2; ++kc)
            for (int e = 0; e < 8; ++e) {
                const int ci = ks * 16 + kc * 8 + e;
                for (int dy = 0; dy < 3; ++dy)
                    for (int dx = 0; dx < 3; ++dx) {
                        const int tp = 3 * dy + dx;
                        __half hi, lo;
                        split(w3[(ci * 3 + dy) * 3 + dx], hi, lo);
                        __half* th = l3 + (size_t)(ks * 2 + 0) * (S::B3TILE / 2);
                        __half* tl = l3 + (size_t)(ks * 2 + 1) * (S::B3TILE / 2);
                        th[(kc * 32 + tp) * 8 + e] = hi;
                        th[(kc * 32 + 9 + tp) * 8 + e] = lo;
                        tl[(kc * 32 + 9 + tp) * 8 + e] = hi;
                    }
            }
}

int launch_cnn_fused(const float* X, long x_ms, const float* U, long u_ms, float* Xout, long o_ms,
                     const float* Bmat, int Nb, int n, int m, int l, const float* b1, const float* b2,
                     const float* b3, const void* wpk, float rs, int n_sm, int* err, cudaStream_t st, UAdvance ua)
{
    switch (m) {
    case 128: return fused_launch<32, 1>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, b2, b3, wpk, rs, n_sm, err, st, ua);
    case 64: return fused_launch<32, 2>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, b2, b3, wpk, rs, n_sm, err, st, ua);
    case 32: return fused_launch<32, 4>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, b2, b3, wpk, rs, n_sm, err, st, ua);
    case 16: return fused_launch<32, 8>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, b1, b2, b3, wpk, rs, n_sm, err, st, ua);
    }
    return 1;
}

}  // namespace oic
