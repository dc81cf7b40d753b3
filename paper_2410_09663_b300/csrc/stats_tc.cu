// stats_tc.cu -- the anomaly products of the sample covariances (Sigma^Y and
// Sigma^XY, ensemble moments with 1/N) on the tcgen05 tensor cores, in one
// pass over the ensemble.
//
//   part2[s][a][c] = sum_{i in split s} sum_j d_i[a][j] e_i[c][j]
//   part1[s][a][j] = sum_{i in split s} d_i[a][j]
//
// with d_i = l_i - l_0 the left rows (the R active state rows, then the p
// perturbed observation rows Y^i = H X^i + V^i) shifted by member 0 and
// e_i = Y^i - Y^0 the observation rows shifted the same way; the
// finalisation removes the mean exactly, C = sum part2 - (1/N) S1_a S1_c^T.
// The member-0 shift keeps every operand at the scale of the anomalies.
//
// FP32 accuracy from TF32 operands: x = hi + lo with hi = tf32(x) and
// lo = tf32(x - hi), so x is carried to ~2^-22; per K step the products
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate in one FP32 tensor-memory
// accumulator (A_lo B_lo, ~2^-22 relative, is dropped).  TF32 keeps FP32's
// exponent range, so no scaling of rows is needed.
//
// Work split: CTA (row tile of 128 left rows, member split).  Eight
// producer warps stream each member's rows of the tile (32 K values a
// stage) into a raw shared-memory ring with cp.async, RD - 1 stages ahead,
// then shift, split, accumulate the S1 sums and store hi / lo into
// 128-byte-swizzled K-major tiles; a loader bulk-copies the member's
// pre-split observation tile; one thread issues the MMAs.  yprep_kernel
// runs first, once per analysis: it writes the observation tiles, the
// shifted observation rows e_i (the producers' source for left rows >= R,
// so every left row is one plain row of some buffer) and the innovations
// D^i = Ybar_t - Y^i.  The issue order is K chunk outer, member inner, so a
// producer keeps the member-0 row values of one chunk in registers.
#include <cuda_fp16.h>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int TM = 128;                                 // left rows per tile (MMA M)
constexpr int KC = 32;                                  // K values per stage: one 128-byte row
constexpr int ST_PW = 8;                                // producer warps
constexpr int ST_LOADER = ST_PW, ST_ISSUER = ST_PW + 1;
constexpr int ST_NT = (ST_PW + 2) * 32;
constexpr int ATILE = TM * 128;                         // one A part (hi or lo), bytes
constexpr long long ST_WAIT = 4000000000LL;             // ~2 s at 2 GHz
constexpr int RD = 4;                                   // raw ring depth (stages)
constexpr int RTILE = TM * 128;                         // one raw stage, bytes

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

// Observation row c of member i, columns j .. j+3 (E row plus noise).
__device__ __forceinline__ float4 yrow4(const float* __restrict__ E, long ms, int m, const RowSet& obs,
                                        const ObsNoise& V, int p, int i, int c, int j)
{
    float4 v = __ldg(reinterpret_cast<const float4*>(E + (long)i * ms + (long)obs.rows[c] * m + j));
    if (V.Va != nullptr) {
        const float* vr = c < V.pa ? V.Va + ((long)i * V.pa + c) * m : V.Vb + ((long)i * (p - V.pa) + (c - V.pa)) * m;
        v = f4add(v, __ldg(reinterpret_cast<const float4*>(vr + j)));
    }
    return v;
}

// One thread per (member, K chunk, observation row c < pp, 16-byte chunk):
// e = Y^i - Y^0 split into the B tile [i][kh][hi rows pp | lo rows pp][128 B]
// (swizzled; zero beyond p and beyond m); for c < p also e itself into
// Ysh [i][c][m] and D^i = Ybar - Y^i.
__global__ void yprep_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet obs, ObsNoise V,
                             const float* __restrict__ Yx, const float* __restrict__ Yu, int n_yx, int KH, int pp,
                             float* __restrict__ Bop, float* __restrict__ Ysh, float* __restrict__ Dbuf)
{
    const int p = obs.count;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long per_member = (long)KH * pp * 8;
    if (e >= (long)N * per_member) return;
    const int i = (int)(e / per_member);
    int rem = (int)(e % per_member);
    const int kh = rem / (pp * 8);
    rem %= pp * 8;
    const int c = rem / 8, k = rem % 8;
    const int j = kh * KC + k * 4;
    float4 hi = make_float4(0.f, 0.f, 0.f, 0.f), lo = hi;
    if (c < p && j < m) {
        const float4 y = yrow4(E, ms, m, obs, V, p, i, c, j);
        const float4 y0 = yrow4(E, ms, m, obs, V, p, 0, c, j);
        const float4 ev = f4sub(y, y0);
        split_tf32(ev, hi, lo);
        *reinterpret_cast<float4*>(Ysh + ((long)i * p + c) * m + j) = ev;
        const float* yb = c < n_yx ? Yx + (long)c * m : Yu + (long)(c - n_yx) * m;
        *reinterpret_cast<float4*>(Dbuf + ((long)i * p + c) * m + j) =
            f4sub(*reinterpret_cast<const float4*>(yb + j), y);
    }
    char* tile = reinterpret_cast<char*>(Bop) + ((size_t)i * KH + kh) * (size_t)(2 * pp) * 128;
    *reinterpret_cast<float4*>(tile + swz(c, k)) = hi;
    *reinterpret_cast<float4*>(tile + swz(pp + c, k)) = lo;
}

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
// instruction descriptor: TF32 A and B (format 2), FP32 D, K-major, N, M
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// a left row's source: member 0's row and the stride between members
// (E rows, or the shifted observation rows, whose member-0 row is zero)
struct RowSrc {
    const float* e;
    long stride;
    bool live;
};

__device__ __forceinline__ float4 load_unit(const RowSrc& s, int i, int j, int m)
{
    if (!s.live || j >= m) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4*>(s.e + (long)i * s.stride + j));
}
// 16 bytes global -> shared, asynchronous; zero-filled when !valid
__device__ __forceinline__ void cp16(uint32_t dst, const float* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// ring of S stages: [A hi 16 KB][A lo 16 KB][B 2 pp x 128 B], 1024-aligned,
// then the raw ring (RD x 16 KB), then the barriers
__global__ void __launch_bounds__(ST_NT, 1)
stats_tc_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet act, RowSet obs,
                const float* __restrict__ Ysh, const float* __restrict__ Bop, int pp, int KH, int S, int splits,
                int tmem_cols, float* __restrict__ part1, float* __restrict__ part2, int* __restrict__ err)
{
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t s0 = (raw + 1023u) & ~1023u;                     // swizzle atoms need 1024-byte alignment
    unsigned char* smem = smem_raw + (s0 - raw);
    const int R = act.count, p = obs.count, M = R + p;
    const int STAGE = 2 * ATILE + 2 * pp * 128;
    const uint32_t rawring = s0 + S * STAGE;
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + S * STAGE + RD * RTILE);   // full bful free done
    uint64_t* full = mb;
    uint64_t* bful = mb + S;
    uint64_t* freeb = mb + 2 * S;
    uint64_t* done = mb + 3 * S;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mb + 3 * S + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int rt = blockIdx.x, sidx = blockIdx.y;
    const int i0 = (int)((long)sidx * N / splits), i1 = (int)((long)(sidx + 1) * N / splits);
    const int nmem = i1 - i0;
    const int nst = KH * nmem;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc::mbar_init(full + s, ST_PW);
            tc::mbar_init(bful + s, 1);
            tc::mbar_init(freeb + s, 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
    }
    if (warp == ST_LOADER) {
        tc::tmem_alloc(tmem_holder, (uint32_t)tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    bool failed = false;

    if (warp < ST_PW) {
        // ---- producers: thread -> 16-byte chunk k of rows rb + 32 u
        const int k = tid & 7, rb = tid >> 3;
        RowSrc src[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = rt * TM + rb + 32 * u;
            src[u].live = a < M;
            if (a < R) {
                src[u].e = E + (long)act.rows[a] * m;
                src[u].stride = ms;
            } else {
                src[u].e = Ysh + (long)(a < M ? a - R : 0) * m;
                src[u].stride = (long)p * m;
            }
        }
        // raw ring: thread's unit u of stage q at raw(q % RD) + row * 128 + k * 16
        auto issue = [&](int q) {
            if (q < nst) {
                const int kh = q / nmem, i = i0 + (q - kh * nmem), j = kh * KC + k * 4;
                const uint32_t dst = rawring + (q % RD) * RTILE + rb * 128 + k * 16;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool v = src[u].live && j < m;
                    cp16(dst + u * 32 * 128, v ? src[u].e + (long)i * src[u].stride + j : E, v);
                }
            }
            cp_commit();                          // empty groups keep the count uniform
        };
        float4 v0[4], s1[4];
        auto flush = [&](int kh) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = rt * TM + rb + 32 * u, j = kh * KC + k * 4;
                if (a < M && j < m) *reinterpret_cast<float4*>(part1 + ((long)sidx * M + a) * m + j) = s1[u];
            }
        };
#pragma unroll
        for (int q = 0; q < RD - 1; ++q) issue(q);
        for (int q = 0; q < nst; ++q) {
            const int kh = q / nmem, qi = q - kh * nmem;
            const int j = kh * KC + k * 4;
            issue(q + RD - 1);
            if (qi == 0) {
                if (kh > 0) flush(kh - 1);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    v0[u] = load_unit(src[u], 0, j, m);
                    s1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            cp_wait<RD - 1>();                    // this thread's copies of stage q have landed
            float4 cur[4];
            const unsigned char* rq = smem + S * STAGE + (q % RD) * RTILE + rb * 128 + k * 16;
#pragma unroll
            for (int u = 0; u < 4; ++u) cur[u] = *reinterpret_cast<const float4*>(rq + u * 32 * 128);
            const int s = q % S;
            if (q >= S) {
                bool ok = true;
                if (lane == 0) ok = tc::mbar_wait_bounded(freeb + s, (uint32_t)((q / S - 1) & 1), ST_WAIT);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) atomicExch(err, DEV_TIMEOUT);
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
            }
            unsigned char* ah = smem + s * STAGE;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = rb + 32 * u;
                const float4 d = f4sub(cur[u], v0[u]);
                s1[u] = f4add(s1[u], d);
                float4 hi, lo;
                split_tf32(d, hi, lo);
                *reinterpret_cast<float4*>(ah + swz(r, k)) = hi;
                *reinterpret_cast<float4*>(ah + ATILE + swz(r, k)) = lo;
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(full + s);
        }
        cp_wait<0>();
        if (!failed && nst > 0) flush(KH - 1);

        // ---- drain: warps w and w + 4 share TMEM lane quarter w % 4 and
        // take alternate 16-column groups
        bool ok = true;
        if (lane == 0 && !failed) ok = tc::mbar_wait_bounded(done, 0u, ST_WAIT);
        ok = __shfl_sync(0xffffffffu, ok, 0) && !failed;
        if (!ok && lane == 0) atomicExch(err, DEV_TIMEOUT);
        tc::fence_after_sync();
        if (ok) {
            const int quarter = warp & 3;
            const int a = rt * TM + 32 * quarter + lane;
            const uint32_t tl = (uint32_t)(32 * quarter) << 16;
            for (int c0 = (warp >> 2) * 16; c0 < pp; c0 += 32) {
                float v[16];
                tc::tmem_ld16(tmem + tl + c0, v);
                tc::tmem_ld_wait();
                if (a < M) {
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        if (c0 + u < p) part2[((long)sidx * M + a) * p + c0 + u] = nst > 0 ? v[u] : 0.f;
                }
            }
        }
    } else if (warp == ST_LOADER && lane == 0) {
        // ---- loader: observation tile (member i, chunk kh) per stage
        const uint32_t bbytes = (uint32_t)(2 * pp * 128);
        int q = 0;
        for (; q < nst; ++q) {
            const int s = q % S;
            if (q >= S && !tc::mbar_wait_bounded(freeb + s, (uint32_t)((q / S - 1) & 1), ST_WAIT)) {
                atomicExch(err, DEV_TIMEOUT);
                break;
            }
            const int kh = q / nmem, i = i0 + (q - kh * nmem);
            const char* src = reinterpret_cast<const char*>(Bop) + ((size_t)i * KH + kh) * bbytes;
            st_expect_tx(bful + s, bbytes);
            st_bulk(s0 + s * STAGE + 2 * ATILE, src, bbytes, bful + s);
        }
        // the copies in flight land before the CTA leaves
        for (int r = q - S < 0 ? 0 : q - S; r < q; ++r)
            tc::mbar_wait_bounded(bful + r % S, (uint32_t)((r / S) & 1), ST_WAIT);
    } else if (warp == ST_ISSUER && lane == 0) {
        // ---- issuer: per stage 4 K steps of 8, three MMAs each
        const uint32_t id = idesc_tf32(TM, pp);
        for (int q = 0; q < nst; ++q) {
            const int s = q % S;
            const uint32_t par = (uint32_t)((q / S) & 1);
            if (!tc::mbar_wait_bounded(full + s, par, ST_WAIT) || !tc::mbar_wait_bounded(bful + s, par, ST_WAIT)) {
                atomicExch(err, DEV_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            const uint32_t base = s0 + s * STAGE;
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
                const uint32_t ah = sw_desc(base + ks * 32);
                const uint32_t al = sw_desc(base + ATILE + ks * 32);
                const uint32_t bh = sw_desc(base + 2 * ATILE + ks * 32);
                const uint32_t bl = sw_desc(base + 2 * ATILE + pp * 128 + ks * 32);
                st_mma(tmem, ah, bh, id, (q | ks) != 0 ? 1u : 0u);
                st_mma(tmem, ah, bl, id, 1u);
                st_mma(tmem, al, bh, id, 1u);
            }
            tc::mma_commit(freeb + s);
        }
        tc::mma_commit(done);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == ST_LOADER) tc::tmem_dealloc(tmem, (uint32_t)tmem_cols);
}

int st_stages(int pp)
{
    const size_t stage = 2 * (size_t)ATILE + (size_t)2 * pp * 128;
    return 1024 + 3 * stage + RD * RTILE + 256 <= 232448 ? 3 : 2;
}

}  // namespace

int stats_tc_rtiles(int M) { return (M + TM - 1) / TM; }
int stats_tc_pp(int p) { return (p + 15) / 16 * 16; }
int stats_tc_kh(int m) { return (m + KC - 1) / KC; }
// one wave of at most 148 CTAs, and at least ~6 members per split so the
// partial sums stay small next to the products
int stats_tc_splits(int M, int N)
{
    int s = 148 / stats_tc_rtiles(M);
    if (s > N / 6) s = N / 6;
    return s < 1 ? 1 : s;
}
size_t stats_tc_bbytes(int N, int p, int m)
{
    return (size_t)N * stats_tc_kh(m) * 2 * stats_tc_pp(p) * 128 + (size_t)N * p * m * sizeof(float);
}
size_t stats_tc_smem(int p)
{
    const int pp = stats_tc_pp(p);
    return 1024 + (size_t)st_stages(pp) * (2 * (size_t)ATILE + (size_t)2 * pp * 128) + RD * RTILE + 256;
}
bool stats_tc_supported(int m, int p)
{
    return p >= 1 && m >= 4 && m % 4 == 0 && stats_tc_pp(p) <= 256 && stats_tc_smem(p) <= 232448;
}

void launch_stats_tc(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
                     const float* Yu, int n_yx, float* Bop, float* part1, float* part2, float* Dbuf, int splits,
                     int* err, cudaStream_t st)
{
    const int p = obs.count, M = act.count + p, pp = stats_tc_pp(p), KH = stats_tc_kh(m);
    const long nprep = (long)N * KH * pp * 8;
    float* Ysh = Bop + (size_t)N * KH * 2 * pp * 32;      // after the observation tiles
    yprep_kernel<<<(unsigned)((nprep + 255) / 256), 256, 0, st>>>(E, ms, N, m, obs, V, Yx, Yu, n_yx, KH, pp, Bop,
                                                                  Ysh, Dbuf);
    const int S = st_stages(pp);
    const int cols = pp <= 32 ? 32 : pp <= 64 ? 64 : pp <= 128 ? 128 : 256;
    const size_t smem = stats_tc_smem(p);
    cudaFuncSetAttribute(stats_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    stats_tc_kernel<<<dim3(stats_tc_rtiles(M), splits), ST_NT, smem, st>>>(E, ms, N, m, act, obs, Ysh, Bop, pp, KH,
                                                                           S, splits, cols, part1, part2, err);
}

}  // namespace oic
