// conv_tc.cu -- hidden 3x3 conv layers of CNN_theta (Eq. (1)) on the tcgen05
// tensor cores at FP32 accuracy, plus a known-answer check of the tensor path.
//
// FP32 accuracy from fp16 tensor cores: every operand x is split into
// x = hi + lo * 2^-11 (hi, lo fp16), and the layer computes
//   main = A_hi B_hi                      (TMEM columns [0, C))
//   corr = A_hi B_lo + A_lo B_hi          (TMEM columns [C, 2C))
//   out  = main + corr * 2^-11,           error ~ 2^-21 per product,
// with the dropped A_lo B_lo term below FP32 rounding.  A_hi is read once
// for both B_hi and B_lo by stacking [B_hi; B_lo] as one N = 2C operand.
//
// Implicit GEMM: a CTA tile is M = 128 pixels = one image row of 128/m
// members side by side.  Input rows stream through a ring of three shared-
// memory slots; each slot holds the row three times, shifted by one pixel
// left / not / right (zero at each member's edges), so tap (dy, dx) of the
// 3x3 stencil is the K-major operand "slot of row y+dy-1, copy dx".  Per
// output row: 9 taps x C/16 K-steps x 2 MMAs (M = 128, N = 2C and N = C,
// K = 16), accumulating into one of two TMEM accumulators while the other is
// drained (tanh epilogue) and the next input row is staged.  The grid is
// persistent: CTA c streams a contiguous range of (member group, row) tiles.
#include <cuda_fp16.h>

#include <vector>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TILE_M = 128;
constexpr long long WAIT_CYCLES = 4000000000LL;   // about 2 s at 2 GHz

template <int C>
struct ConvTcShape {
    static constexpr int KC = C / 8;                   // 8-channel core-matrix columns
    static constexpr int KS = C / 16;                  // K = 16 steps per tap
    static constexpr int PLANE = TILE_M * 16;          // 128 pixels x 8 fp16
    static constexpr int PART = KC * PLANE;            // one (copy, hi|lo) of a row
    static constexpr int SLOT = 3 * 2 * PART;          // 3 shifted copies x {hi, lo}
    static constexpr int BTILE = 2 * (2 * C) * 16;     // one (tap, K-step) weight tile
    static constexpr int BBYTES = 9 * KS * BTILE;
    static constexpr int OFF_B = 3 * SLOT;
    static constexpr int OFF_MISC = OFF_B + BBYTES;    // mbarrier, TMEM base, bias
    // 8 KB of slack past the last operand keeps every descriptor walk inside
    // the CTA's shared memory even for a misread stride
    static constexpr int SMEM = OFF_MISC + 64 + C * 4 + 8192;
    static constexpr int TMEM_COLS = 4 * C >= 32 ? 4 * C : 32;   // two accumulators of 2C
    static constexpr int CHUNKS = TILE_M * KC / TC_THREADS;       // 16-byte chunks per thread
};

__device__ __forceinline__ int slot_of(int r) { return ((r % 3) + 3) % 3; }

// Reads one input row (FP32, channel-planar activations) for the member group
// into registers: each thread owns CHUNKS (pixel, 8-channel) chunks.
template <int C>
__device__ __forceinline__ void fetch_row(float (&v)[ConvTcShape<C>::CHUNKS][8], const float* __restrict__ in,
                                          int Nb, int n, int m, int g, int r)
{
    using S = ConvTcShape<C>;
    const int G = TILE_M / m;
#pragma unroll
    for (int i = 0; i < S::CHUNKS; ++i) {
        const int chunk = threadIdx.x + TC_THREADS * i;
        const int px = chunk % TILE_M, kc = chunk / TILE_M;
        const int mb = g * G + px / m, x = px % m;
        const bool ok = r >= 0 && r < n && mb < Nb;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            v[i][c] = ok ? __ldg(in + (((long)mb * C + kc * 8 + c) * n + r) * m + x) : 0.f;
    }
}

// Splits the fetched row into hi/lo fp16 and writes the three shifted copies
// into `slot` (copy d holds pixel x + d - 1 of the same member, zero off the edge).
template <int C>
__device__ __forceinline__ void store_row(const float (&v)[ConvTcShape<C>::CHUNKS][8], unsigned char* slot, int m)
{
    using S = ConvTcShape<C>;
#pragma unroll
    for (int i = 0; i < S::CHUNKS; ++i) {
        const int chunk = threadIdx.x + TC_THREADS * i;
        const int px = chunk % TILE_M, kc = chunk / TILE_M;
        const int x = px % m;
        __align__(16) __half hi[8], lo[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) tc::split_f16(v[i][c], hi[c], lo[c]);
        const uint4 H = *reinterpret_cast<const uint4*>(hi);
        const uint4 L = *reinterpret_cast<const uint4*>(lo);
        const uint4 Z = make_uint4(0u, 0u, 0u, 0u);
        unsigned char* base = slot + kc * S::PLANE;
        auto put = [&](int d, int pos, uint4 h, uint4 l) {
            *reinterpret_cast<uint4*>(base + (d * 2 + 0) * S::PART + pos * 16) = h;
            *reinterpret_cast<uint4*>(base + (d * 2 + 1) * S::PART + pos * 16) = l;
        };
        if (x + 1 < m) put(0, px + 1, H, L);
        if (x == 0) put(0, px, Z, Z);
        put(1, px, H, L);
        if (x >= 1) put(2, px - 1, H, L);
        if (x == m - 1) put(2, px, Z, Z);
    }
}

template <int C>
__device__ __forceinline__ void issue_row_mmas(unsigned char* smem, uint32_t acc, int y)
{
    using S = ConvTcShape<C>;
    const uint32_t s0 = tc::smem_u32(smem);
    constexpr uint32_t id1 = tc::idesc_f16(TILE_M, 2 * C);
    constexpr uint32_t id2 = tc::idesc_f16(TILE_M, C);
    uint32_t accumulate = 0;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const uint32_t slot = s0 + slot_of(y + dy - 1) * S::SLOT;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
            for (int ks = 0; ks < S::KS; ++ks) {
                const uint32_t a_hi = slot + (dx * 2 + 0) * S::PART + 2 * ks * S::PLANE;
                const uint32_t a_lo = slot + (dx * 2 + 1) * S::PART + 2 * ks * S::PLANE;
                const uint32_t b = s0 + S::OFF_B + ((dy * 3 + dx) * S::KS + ks) * S::BTILE;
                const uint64_t da_hi = tc::desc_kmajor(a_hi, S::PLANE, 128);
                const uint64_t da_lo = tc::desc_kmajor(a_lo, S::PLANE, 128);
                const uint64_t db = tc::desc_kmajor(b, 2 * C * 16, 128);
                tc::mma_f16(acc, da_hi, db, id1, accumulate);
                tc::mma_f16(acc + C, da_lo, db, id2, 1u);
                accumulate = 1;
            }
        }
    }
}

// out[b] = tanh(conv(in[b]) + bias) for a C -> C layer.
template <int C>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv_tc_split_kernel(const float* __restrict__ in, float* __restrict__ out, const __half* __restrict__ wpk,
                     const float* __restrict__ bias, int Nb, int n, int m, int* __restrict__ err)
{
    pdl_begin();
    using S = ConvTcShape<C>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MISC);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(smem + S::OFF_MISC + 8);
    float* sbias = reinterpret_cast<float*>(smem + S::OFF_MISC + 64);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    // weights -> shared memory (already in the MMA operand layout)
    {
        const uint4* src = reinterpret_cast<const uint4*>(wpk);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::OFF_B);
        for (int e = tid; e < S::BBYTES / 16; e += TC_THREADS) dst[e] = src[e];
        for (int e = tid; e < C; e += TC_THREADS) sbias[e] = bias[e];
    }
    if (tid == 0) {
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

    const int G = TILE_M / m;
    const int groups = (Nb + G - 1) / G;
    const long total = (long)groups * n;
    const long t0 = total * blockIdx.x / gridDim.x, t1 = total * (blockIdx.x + 1) / gridDim.x;
    uint32_t phase = 0;
    int par = 0;
    bool failed = false;
    float pf[S::CHUNKS][8];

    for (long t = t0; t < t1 && !failed;) {
        const int g = (int)(t / n);
        const int y0 = (int)(t % n);
        const long rem = t1 - t;
        const int y1 = (long)(n - y0) < rem ? n : (int)(y0 + rem);
        t += y1 - y0;
        // prologue: rows y0-1, y0, y0+1
        for (int r = y0 - 1; r <= y0 + 1; ++r) {
            fetch_row<C>(pf, in, Nb, n, m, g, r);
            store_row<C>(pf, smem + slot_of(r) * S::SLOT, m);
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_row_mmas<C>(smem, tmem + par * 2 * C, y0);
            tc::mma_commit(mbar);
        }
        if (y0 + 1 < y1) fetch_row<C>(pf, in, Nb, n, m, g, y0 + 2);
        for (int y = y0; y < y1; ++y) {
            const bool ok = tc::mbar_wait_bounded(mbar, phase, WAIT_CYCLES);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            if (y + 1 < y1) {
                store_row<C>(pf, smem + slot_of(y + 2) * S::SLOT, m);
                tc::fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc::fence_after_sync();
                    issue_row_mmas<C>(smem, tmem + (par ^ 1) * 2 * C, y + 1);
                    tc::mma_commit(mbar);
                }
                if (y + 2 < y1) fetch_row<C>(pf, in, Nb, n, m, g, y + 3);
            }
            // epilogue of row y: warp w reads TMEM lanes 32 (w % 4) .., channels
            // (w / 4) * C/2 .. of main and corr
            {
                const int q = warp & 3, h = warp >> 2;
                const uint32_t lane_addr = (uint32_t)(32 * q) << 16;
                const uint32_t col = par * 2 * C + h * (C / 2);
                float mv[16], cv[16];
                tc::tmem_ld16(tmem + lane_addr + col, mv);
                tc::tmem_ld16(tmem + lane_addr + col + C, cv);
                tc::tmem_ld_wait();
                const int px = 32 * q + lane;
                const int mb = g * G + px / m, x = px % m;
                if (mb < Nb) {
#pragma unroll
                    for (int j = 0; j < C / 2; ++j) {
                        const int co = h * (C / 2) + j;
                        const float val = fmaf(cv[j], tc::SPLIT_INV, mv[j]) + sbias[co];
                        out[(((long)mb * C + co) * n + y) * m + x] = tanhf(val);
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            par ^= 1;
        }
    }
    if (failed) {
        if (tid == 0) atomicExch(err, DEV_TIMEOUT);
        // give any MMA still in flight a last bounded chance to land before
        // the tensor memory is released
        tc::mbar_wait_bounded(mbar, phase, WAIT_CYCLES);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

// ---------------------------------------------------------------- self-test
// D = A B^T with M = 128, K = 32, N = 64, then D[:, 32:64] += A B[0:32]^T,
// on small integers (exact in fp16 and fp32); every element is checked
// against a CUDA-core dot product.  res[0] = mismatches (-1: timeout),
// res[1..4] = first mismatch (row, col, got, want).
__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(int* __restrict__ res)
{
    pdl_begin();
    constexpr int M = 128, N = 64, K = 32;
    // operands use (K/8)*M*16 and (K/8)*N*16 bytes; the arrays are larger so a
    // misread stride still reads inside the CTA's shared memory
    __shared__ __align__(1024) unsigned char As[32 * 1024];
    __shared__ __align__(1024) unsigned char Bs[8 * 1024];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    auto aval = [](int r, int k) { return (float)((r * 3 + k * 7) % 11 - 5); };
    auto bval = [](int c, int k) { return (float)((c * 5 + k * 3) % 9 - 4); };
    for (int e = tid; e < M * K; e += 128) {
        const int r = e / K, k = e % K;
        reinterpret_cast<__half*>(As + (k / 8) * M * 16 + r * 16)[k % 8] = __float2half(aval(r, k));
    }
    for (int e = tid; e < N * K; e += 128) {
        const int c = e / K, k = e % K;
        reinterpret_cast<__half*>(Bs + (k / 8) * N * 16 + c * 16)[k % 8] = __float2half(bval(c, k));
    }
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_holder, 512);      // all columns: any N stays inside
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_holder;
    if (tid == 0) {
        const uint32_t a = tc::smem_u32(As), b = tc::smem_u32(Bs);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t da = tc::desc_kmajor(a + 2 * ks * M * 16, M * 16, 128);
            const uint64_t db = tc::desc_kmajor(b + 2 * ks * N * 16, N * 16, 128);
            tc::mma_f16(tmem, da, db, tc::idesc_f16(M, N), ks > 0);
        }
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t da = tc::desc_kmajor(a + 2 * ks * M * 16, M * 16, 128);
            const uint64_t db = tc::desc_kmajor(b + 2 * ks * N * 16, N * 16, 128);
            tc::mma_f16(tmem + 32, da, db, tc::idesc_f16(M, 32), 1u);
        }
        tc::mma_commit(&mbar);
    }
    const bool ok = tc::mbar_wait_bounded(&mbar, 0, WAIT_CYCLES);
    tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) atomicExch(res, -1);
    } else {
        const int r = 32 * warp + lane;
        int bad = 0;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
            tc::tmem_ld_wait();
            for (int j = 0; j < 16; ++j) {
                const int c = c0 + j;
                float want = 0.f;
                for (int k = 0; k < K; ++k) want += aval(r, k) * bval(c, k);
                if (c >= 32)
                    for (int k = 0; k < K; ++k) want += aval(r, k) * bval(c - 32, k);
                if (v[j] != want) {
                    if (atomicAdd(res, 1) == 0) {
                        res[1] = r; res[2] = c; res[3] = (int)v[j]; res[4] = (int)want;
                    }
                    ++bad;
                }
            }
        }
        (void)bad;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

bool conv_tc_supported(int cin, int cout, int m)
{
    return cin == 32 && cout == 32 && m >= 8 && m <= TILE_M && TILE_M % m == 0;
}

size_t conv_tc_packed_bytes(int C)
{
    return C == 32 ? (size_t)ConvTcShape<32>::BBYTES : 0;
}

void conv_tc_pack_weights(const float* w, int C, void* dst_host)
{
    const int KS = C / 16;
    __half* out = static_cast<__half*>(dst_host);
    for (int dy = 0; dy < 3; ++dy)
        for (int dx = 0; dx < 3; ++dx)
            for (int ks = 0; ks < KS; ++ks)
                for (int kc = 0; kc < 2; ++kc)
                    for (int r = 0; r < 2 * C; ++r)
                        for (int e = 0; e < 8; ++e) {
                            const int ci = ks * 16 + kc * 8 + e, co = r % C;
                            const float v = w[((co * C + ci) * 3 + dy) * 3 + dx];
                            const __half hi = __float2half_rn(v);
                            const __half lo = __float2half_rn((v - __half2float(hi)) * tc::SPLIT_SCALE);
                            const size_t idx = ((((size_t)(dy * 3 + dx) * KS + ks) * 2 + kc) * (2 * C) + r) * 8 + e;
                            out[idx] = r < C ? hi : lo;
                        }
}

int conv_tc_configure()
{
    using S = ConvTcShape<32>;
    return cudaFuncSetAttribute(conv_tc_split_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                S::SMEM) == cudaSuccess
               ? 0
               : 1;
}

void launch_conv_tc(const float* in, float* out, const void* wpk, const float* bias, int C, int Nb, int n,
                    int m, int n_sm, int* err, cudaStream_t st)
{
    using S = ConvTcShape<32>;
    (void)C;
    const int G = TILE_M / m;
    const long tiles = (long)((Nb + G - 1) / G) * n;
    const int grid = (int)(tiles < n_sm ? tiles : n_sm);
    pdl_launch(conv_tc_split_kernel<32>, grid, TC_THREADS, S::SMEM, st, in, out, static_cast<const __half*>(wpk),
                                                               bias, Nb, n, m, err);
}

void launch_tc_selftest(int* res, cudaStream_t st)
{
    pdl_launch(tc_selftest_kernel, 1, 128, 0, st, res);
}

}  // namespace oic
