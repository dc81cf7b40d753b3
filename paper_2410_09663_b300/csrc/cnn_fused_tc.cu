// cnn_fused_tc.cu -- the whole surrogate X_{t+1} = X_t + s * CNN_theta(X_t, U_t)
// of Eq. (1), structure [X; B U] -> C (tanh) -> C (tanh) -> 1, in ONE kernel:
//
//   first layer (2 -> C, tanh)   CUDA cores, computed row by row as the
//                                operand producer of the hidden layer
//   hidden layer (C -> C, tanh)  tcgen05 tensor cores, FP32-accurate fp16
//                                split (main = A_hi B_hi, corr = A_hi B_lo +
//                                A_lo B_hi, out = main + corr 2^-11)
//   last layer (C -> 1) + residual  CUDA cores, as rolling per-pixel partial
//                                sums over the three stencil rows
//
// Only X, U and the weights are read and X_next written; no activation
// leaves the SM.  A CTA owns a group of G = 128/m members; an M = 128 tile is
// one image row of the group with the members INTERLEAVED pixel by pixel
// (position G + G x + b for member b, pixel x, zero pads at both ends).  A
// shift of the stencil by one pixel is then a shift of the operand start by
// G positions = 16 G bytes, so one copy of each activation row serves all
// three horizontal taps, and members never see each other's pixels.  Rows
// stream through a ring of three operand slots; the tensor core works on
// hidden row r while the CUDA cores produce first-layer row r+2 and drain
// hidden row r-1.  The grid is persistent over contiguous (group, row) ranges.
#include <cuda_fp16.h>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int FT = 512;                                 // threads (16 warps)
constexpr int FM = 128;                                 // tile rows (pixels)
constexpr long long F_WAIT = 4000000000LL;

__host__ __device__ constexpr int al16(int x) { return (x + 15) / 16 * 16; }

template <int C, int G>
struct FS {
    static constexpr int KC = C / 8, KS = C / 16;
    static constexpr int NPOS = FM + 2 * G;             // operand positions incl. pads
    static constexpr int PLANE = NPOS * 16;             // one (part, 8-channel) plane
    static constexpr int SLOT = 2 * KC * PLANE;         // hi and lo of one activation row
    static constexpr int BTILE = 2 * (2 * C) * 16;
    static constexpr int BBYTES = 9 * KS * BTILE;
    static constexpr int SP = NPOS | 1;                 // odd FP32 row stride (bank spread)
    static constexpr int NXB = 6;                       // ring of [X; B U] rows
    static constexpr int OFF_SLOT = 0;
    static constexpr int OFF_B = OFF_SLOT + 3 * SLOT;
    static constexpr int OFF_H2 = OFF_B + BBYTES;                      // [C][SP] fp32
    static constexpr int OFF_XB = OFF_H2 + al16(C * SP * 4);           // [NXB][2][SP] fp32
    static constexpr int OFF_W1 = OFF_XB + al16(NXB * 2 * SP * 4);     // [C/8][2][9][8]
    static constexpr int OFF_B1 = OFF_W1 + al16(C * 2 * 9 * 4);
    static constexpr int OFF_W3 = OFF_B1 + al16(C * 4);                // [C/4][4][12] (9 used)
    static constexpr int OFF_B2 = OFF_W3 + al16(C * 12 * 4);
    static constexpr int OFF_MISC = OFF_B2 + al16(C * 4);              // b3, mbar, tmem
    static constexpr int OFF_DYN = OFF_MISC + 64;                      // U group, B matrix
    static constexpr int TMEM_COLS = 4 * C;
};

__device__ __forceinline__ int mod_pos(int r, int k) { return ((r % k) + k) % k; }

// tanh(x) = 1 - 2 / (1 + e^{2x}): saturates correctly at both ends; absolute
// error a few 1e-7 (the exponential and the quotient are each within a few
// ulps), which is below the FP32 rounding of the layer's inputs.
__device__ __forceinline__ float tanh_fast(float x)
{
    return 1.f - __fdividef(2.f, 1.f + __expf(2.f * x));
}

template <int C, int G>
__device__ __forceinline__ void issue_hidden_mmas(uint32_t s0, uint32_t acc, int r)
{
    using S = FS<C, G>;
    constexpr uint32_t id1 = tc::idesc_f16(FM, 2 * C);
    constexpr uint32_t id2 = tc::idesc_f16(FM, C);
    uint32_t accumulate = 0;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const uint32_t slot = s0 + S::OFF_SLOT + mod_pos(r + dy - 1, 3) * S::SLOT;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                // tap dx reads positions shifted by (dx - 1) G, i.e. start + dx G 16 bytes
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
__global__ void __launch_bounds__(FT, 1)
cnn_fused_kernel(const float* __restrict__ X, long x_ms, const float* __restrict__ U, long u_ms,
                 float* __restrict__ Xout, long o_ms, const float* __restrict__ Bmat, int Nb, int n, int l,
                 const float* __restrict__ w1, const float* __restrict__ b1, const __half* __restrict__ wpk2,
                 const float* __restrict__ b2, const float* __restrict__ w3, const float* __restrict__ b3,
                 float rs, int* __restrict__ err)
{
    using S = FS<C, G>;
    static_assert(C == 32, "one 16-byte chunk of 8 channels per producer thread");
    constexpr int m = FM / G;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* h2 = reinterpret_cast<float*>(smem + S::OFF_H2);
    float* xb = reinterpret_cast<float*>(smem + S::OFF_XB);
    float* sw1 = reinterpret_cast<float*>(smem + S::OFF_W1);
    float* sb1 = reinterpret_cast<float*>(smem + S::OFF_B1);
    float* sw3 = reinterpret_cast<float*>(smem + S::OFF_W3);
    float* sb2 = reinterpret_cast<float*>(smem + S::OFF_B2);
    float* sb3 = reinterpret_cast<float*>(smem + S::OFF_MISC);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MISC + 16);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::OFF_MISC + 32);
    float* su = reinterpret_cast<float*>(smem + S::OFF_DYN);                 // [G][l][m]
    float* sB = su + G * l * m;                                              // [n][l]
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const uint32_t s0 = tc::smem_u32(smem);

    // ---- one-time set-up: zero the operand ring (its pads stay zero), copy weights
    for (int e = tid; e < (S::OFF_B - S::OFF_SLOT) / 16; e += FT)
        reinterpret_cast<uint4*>(smem + S::OFF_SLOT)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < S::BBYTES / 16; e += FT)
        reinterpret_cast<uint4*>(smem + S::OFF_B)[e] = reinterpret_cast<const uint4*>(wpk2)[e];
    for (int e = tid; e < C * S::SP; e += FT) h2[e] = 0.f;
    for (int e = tid; e < S::NXB * 2 * S::SP; e += FT) xb[e] = 0.f;
    for (int e = tid; e < C * 18; e += FT) {     // [co][ch][tap] -> [co/8][ch][tap][co%8]
        const int co = e / 18, r = e % 18;
        sw1[((co / 8) * 18 + r) * 8 + (co % 8)] = w1[e];
    }
    // last-layer weights as [j][quarter][12]: channel ci = quarter * C/4 + j, so
    // the four channel quarters read by one warp fall in different banks
    for (int e = tid; e < C * 12; e += FT) {
        const int slot = e / 12, k = e % 12;
        const int j = slot / 4, qq = slot % 4, ci = qq * (C / 4) + j;
        sw3[e] = k < 9 ? w3[ci * 9 + k] : 0.f;
    }
    for (int e = tid; e < C; e += FT) { sb1[e] = b1[e]; sb2[e] = b2[e]; }
    for (int e = tid; e < n * l; e += FT) sB[e] = Bmat[e];
    if (tid == 0) {
        sb3[0] = b3[0];
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_holder, S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    const int groups = (Nb + G - 1) / G;
    const long total = (long)groups * n;
    const long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    uint32_t phase = 0;
    int par = 0;
    bool failed = false;

    // roles: producer = (pixel pp, 8-channel chunk cq); last layer = (pixel
    // lp, 8-channel quarter lq); epilogue = (TMEM lane quarter, channel group)
    const int pp = tid % FM, cq = tid / FM;
    const int lp = tid >> 2, lq = tid & 3;

    for (long t = t0; t < t1 && !failed;) {
        const int g = (int)(t / n);
        const int ys = (int)(t % n);
        const long rem = t1 - t;
        const int ye = (long)(n - ys) < rem ? n : (int)(ys + rem);
        t += ye - ys;
        const int r_lo = ys > 0 ? ys - 1 : 0;
        const int r_hi = ye < n ? ye : n - 1;

        for (int e = tid; e < G * l * m; e += FT) {
            const int b = e / (l * m), rr = e % (l * m);
            const int mb = g * G + b;
            su[e] = mb < Nb ? U[(long)mb * u_ms + rr] : 0.f;
        }
        __syncthreads();

        // [X; B U] row r into its ring slot (zero outside the image / group)
        auto load_xb = [&](int r) {
            if (tid < FM) {
                float* d = xb + mod_pos(r, S::NXB) * 2 * S::SP;
                const int b = tid / m, x = tid % m;     // coalesced over x
                const int mb = g * G + b;
                const int q = G + G * x + b;
                float xv = 0.f, bu = 0.f;
                if (r >= 0 && r < n && mb < Nb) {
                    xv = X[(long)mb * x_ms + (long)r * m + x];
                    const float* ub = su + b * l * m + x;
                    for (int c = 0; c < l; ++c) bu = fmaf(sB[r * l + c], ub[c * m], bu);
                }
                d[q] = xv;
                d[S::SP + q] = bu;
            }
        };
        // first layer row r, this thread's 8 channels of pixel pp -> hi/lo fp16
        auto first_layer = [&](int r, uint4& hv, uint4& lv) {
            if (r >= 0 && r < n) {
                float acc[8];
                const float4 bA = *reinterpret_cast<const float4*>(sb1 + 8 * cq);
                const float4 bB = *reinterpret_cast<const float4*>(sb1 + 8 * cq + 4);
                acc[0] = bA.x; acc[1] = bA.y; acc[2] = bA.z; acc[3] = bA.w;
                acc[4] = bB.x; acc[5] = bB.y; acc[6] = bB.z; acc[7] = bB.w;
                const int q = G + pp;
                const float* wq = sw1 + cq * 18 * 8;
#pragma unroll
                for (int dy = 0; dy < 3; ++dy) {
                    const float* row = xb + mod_pos(r + dy - 1, S::NXB) * 2 * S::SP;
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch) {
                        const float v3[3] = {row[ch * S::SP + q - G], row[ch * S::SP + q], row[ch * S::SP + q + G]};
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const float* w = wq + (ch * 9 + dy * 3 + dx) * 8;
                            const float4 wa = *reinterpret_cast<const float4*>(w);
                            const float4 wb = *reinterpret_cast<const float4*>(w + 4);
                            const float v = v3[dx];
                            acc[0] = fmaf(wa.x, v, acc[0]); acc[1] = fmaf(wa.y, v, acc[1]);
                            acc[2] = fmaf(wa.z, v, acc[2]); acc[3] = fmaf(wa.w, v, acc[3]);
                            acc[4] = fmaf(wb.x, v, acc[4]); acc[5] = fmaf(wb.y, v, acc[5]);
                            acc[6] = fmaf(wb.z, v, acc[6]); acc[7] = fmaf(wb.w, v, acc[7]);
                        }
                    }
                }
                __align__(16) __half hi[8], lo[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) tc::split_f16(tanh_fast(acc[e]), hi[e], lo[e]);
                hv = *reinterpret_cast<const uint4*>(hi);
                lv = *reinterpret_cast<const uint4*>(lo);
            } else {
                hv = lv = make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto store_h1 = [&](int r, const uint4& hv, const uint4& lv) {
            unsigned char* slot = smem + S::OFF_SLOT + mod_pos(r, 3) * S::SLOT;
            const int q = G + pp;
            *reinterpret_cast<uint4*>(slot + cq * S::PLANE + q * 16) = hv;
            *reinterpret_cast<uint4*>(slot + (S::KC + cq) * S::PLANE + q * 16) = lv;
        };

        // prologue: [X; B U] rows r_lo-2 .. r_lo+3, first-layer rows r_lo-1 .. r_lo+1
        for (int r = r_lo - 2; r <= r_lo + 3; ++r) load_xb(r);
        __syncthreads();
        for (int r = r_lo - 1; r <= r_lo + 1; ++r) {
            uint4 hv, lv;
            first_layer(r, hv, lv);
            store_h1(r, hv, lv);
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_hidden_mmas<C, G>(s0, tmem + par * 2 * C, r_lo);
            tc::mma_commit(mbar);
        }
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;            // outputs of rows r-1, r, r+1
        for (int r = r_lo; r <= r_hi; ++r) {
            const bool more = r + 1 <= r_hi;
            uint4 hv, lv;
            if (more) first_layer(r + 2, hv, lv);      // overlaps hidden row r on the tensor core
            const bool ok = tc::mbar_wait_bounded(mbar, phase, F_WAIT);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            if (more) {
                store_h1(r + 2, hv, lv);
                tc::fence_proxy_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after_sync();
                    issue_hidden_mmas<C, G>(s0, tmem + (par ^ 1) * 2 * C, r + 1);
                    tc::mma_commit(mbar);
                }
                load_xb(r + 4);                          // slot of row r - 2, no longer read
            } else {
                tc::fence_before_sync();
                __syncthreads();                        // previous row's last layer is done with h2
            }
            // hidden row r: tanh(main + corr 2^-11 + b2) -> h2[co][G + lane]
            {
                const int q4 = warp & 3, cg = warp >> 2;  // lane quarter, 8-channel group
                const uint32_t taddr = tmem + ((uint32_t)(32 * q4) << 16) + par * 2 * C + cg * 8;
                float mv[8], cv[8];
                tmem_ld8(taddr, mv);
                tmem_ld8(taddr + C, cv);
                tc::tmem_ld_wait();
                const int pos = G + 32 * q4 + lane;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int co = cg * 8 + j;
                    h2[co * S::SP + pos] = tanh_fast(fmaf(cv[j], tc::SPLIT_INV, mv[j]) + sb2[co]);
                }
            }
            __syncthreads();
            // last layer: contributions of hidden row r to output rows r+1, r, r-1
            {
                const int q = G + lp;
                float p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll
                for (int j = 0; j < C / 4; ++j) {
                    const int ci = lq * (C / 4) + j;
                    const float* hrow = h2 + ci * S::SP;
                    const float v0 = hrow[q - G], v1 = hrow[q], v2 = hrow[q + G];
                    const float* wr = sw3 + (j * 4 + lq) * 12;
                    const float4 wA = *reinterpret_cast<const float4*>(wr);
                    const float4 wB = *reinterpret_cast<const float4*>(wr + 4);
                    const float w8 = wr[8];
                    p0 = fmaf(wA.x, v0, fmaf(wA.y, v1, fmaf(wA.z, v2, p0)));
                    p1 = fmaf(wA.w, v0, fmaf(wB.x, v1, fmaf(wB.y, v2, p1)));
                    p2 = fmaf(wB.z, v0, fmaf(wB.w, v1, fmaf(w8, v2, p2)));
                }
                p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
                p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
                p2 += __shfl_xor_sync(0xffffffffu, p2, 1);
                p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
                p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
                p2 += __shfl_xor_sync(0xffffffffu, p2, 2);
                a0 += p2;                               // kernel row 2 of hidden row r -> output r-1
                a1 += p1;
                a2 += p0;
                const int ro = r - 1;
                if (lq == 0 && ro >= ys && ro < ye) {
                    const int b = lp % G, x = lp / G, mb = g * G + b;
                    if (mb < Nb) {
                        const float xv = xb[mod_pos(ro, S::NXB) * 2 * S::SP + q];
                        Xout[(long)mb * o_ms + (long)ro * m + x] = fmaf(rs, a0 + sb3[0], xv);
                    }
                }
                a0 = a1; a1 = a2; a2 = 0.f;
            }
            par ^= 1;
        }
        if (!failed && ye == n && n - 1 >= ys && lq == 0) {
            // bottom row: the hidden row below the image is zero
            const int b = lp % G, x = lp / G, mb = g * G + b;
            if (mb < Nb) {
                const float xv = xb[mod_pos(n - 1, S::NXB) * 2 * S::SP + G + lp];
                Xout[(long)mb * o_ms + (long)(n - 1) * m + x] = fmaf(rs, a0 + sb3[0], xv);
            }
        }
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicExch(err, DEV_TIMEOUT);
        tc::mbar_wait_bounded(mbar, phase, F_WAIT);
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
                 const float* Bmat, int Nb, int n, int l, const float* w1, const float* b1, const void* wpk2,
                 const float* b2, const float* w3, const float* b3, float rs, int n_sm, int* err,
                 cudaStream_t st)
{
    const size_t smem = fused_smem<C, G>(n, l);
    if (smem > 227 * 1024) return 1;
    static size_t configured = 0;                 // largest size the attribute allows so far
    if (smem > configured) {
        if (cudaFuncSetAttribute(cnn_fused_kernel<C, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024) != cudaSuccess)
            return 1;
        configured = 227 * 1024;
    }
    const long tiles = (long)((Nb + G - 1) / G) * n;
    const int grid = (int)(tiles < n_sm ? tiles : n_sm);
    cnn_fused_kernel<C, G><<<grid, FT, smem, st>>>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, w1, b1,
                                                  static_cast<const __half*>(wpk2), b2, w3, b3, rs, err);
    return 0;
}

}  // namespace

bool cnn_fused_supported(int n_layers, const int* channels, int n, int m, int l)
{
    if (n_layers != 3 || channels[1] != 32 || channels[2] != 32) return false;
    if (!(m == 16 || m == 32 || m == 64 || m == 128)) return false;
    const int G = FM / m;
    const size_t dyn = sizeof(float) * ((size_t)G * l * m + (size_t)n * l);
    return dyn <= 48 * 1024;                      // keeps the whole layout under 227 KB
}

int launch_cnn_fused(const float* X, long x_ms, const float* U, long u_ms, float* Xout, long o_ms,
                     const float* Bmat, int Nb, int n, int m, int l, const float* w1, const float* b1,
                     const void* wpk2, const float* b2, const float* w3, const float* b3, float rs, int n_sm,
                     int* err, cudaStream_t st)
{
    switch (m) {
    case 128: return fused_launch<32, 1>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, w1, b1, wpk2, b2, w3, b3, rs, n_sm, err, st);
    case 64: return fused_launch<32, 2>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, w1, b1, wpk2, b2, w3, b3, rs, n_sm, err, st);
    case 32: return fused_launch<32, 4>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, w1, b1, wpk2, b2, w3, b3, rs, n_sm, err, st);
    case 16: return fused_launch<32, 8>(X, x_ms, U, u_ms, Xout, o_ms, Bmat, Nb, n, l, w1, b1, wpk2, b2, w3, b3, rs, n_sm, err, st);
    }
    return 1;
}

}  // namespace oic
