// stats_tc.cu -- the anomaly products of the sample covariances (Sigma^Y and
// Sigma^XY, ensemble moments with 1/N) on the tcgen05 tensor cores, in one
// pass over the ensemble.
//
//   part2[s][a][c] = sum_{i in split s} sum_j d_i[a][j] e_i[c][j]
//   part1[s][a][j] = sum_{i in split s} d_i[a][j]
//
// with d_i = l_i - l_0 the left rows (the R active state rows, then the p
// perturbed observation rows Y^i = H X^i + V^i) shifted by member 0 and
// e_i = Y^i - H X^0 the observation rows shifted by member 0's unperturbed
// value (any shift constant over the members gives the same moments; this
// one needs no draw of member 0's perturbation); the finalisation removes
// the mean exactly, C = sum part2 - (1/N) S1_a S1_c^T.  The shift keeps
// every operand at the scale of the anomalies and the perturbations.
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
// pre-split observation tile; one warp (an elected lane) issues the MMAs.  yprep_kernel
// runs first, once per analysis: it writes the observation tiles, the
// shifted observation rows e_i (the producers' source for left rows >= R,
// so every left row is one plain row of some buffer) and the innovations
// D^i = Ybar_t - Y^i.  The issue order is K chunk outer, member inner, so a
// producer keeps the member-0 row values of one chunk in registers.
#include <cuda_fp16.h>

#include "oic_internal.cuh"
#include "tc_sm103.cuh"
#include "tc_tf32.cuh"

namespace oic {
namespace {

using namespace tf32;

constexpr int TM = 128;                                 // left rows per tile (MMA M)
constexpr int KC = 32;                                  // K values per stage: one 128-byte row
constexpr int ST_PW = 8;                                // producer warps
constexpr int ST_LOADER = ST_PW, ST_ISSUER = ST_PW + 1;
constexpr int ST_NT = (ST_PW + 2) * 32;
constexpr int ATILE = TM * 128;                         // one A part (hi or lo), bytes
constexpr long long ST_WAIT = 4000000000LL;             // ~2 s at 2 GHz
constexpr int RD = 4;                                   // raw ring depth (stages)
constexpr int RTILE = TM * 128;                         // one raw stage, bytes

// V^i of observation row c, columns j .. j+3 (zero on the constraint rows,
// whose perturbation is already in E, and without a live noise source).
__device__ __forceinline__ float4 obs_noise4(const ObsNoise& V, const RowSet& obs, int p, int i, int c, int j, int m)
{
    if (!V.a.live() || c >= p - obs.nc) return make_float4(0.f, 0.f, 0.f, 0.f);
    return c < V.pa ? noise4(V.a, ((long)i * V.pa + c) * m + j)
                    : noise4(V.b, ((long)i * (p - obs.nc - V.pa) + (c - V.pa)) * m + j);
}

// One block per (member i, K chunk kh of 32 columns j); thread units
// (observation row c < pp, 16-byte chunk): e = Y^i - H X^0 split into the B
// tile [i][kh][hi rows pp | lo rows pp][128 B] (swizzled; zero beyond p and
// beyond m); for c < p also e itself into Ysh [i][c][m].  The innovations
// D^i = Ybar - Y^i (Ybar = 0 on the obs.nc trailing constraint rows, whose
// perturbation is already in E) go either plainly to Dbuf [i][c][m] or, through a
// transpose in shared memory, to the member update's operand Bd: rows
// n = i m + j, K = c in chunks of 32, [kc][hi | lo][N m rows][128 B]
// (swizzled, zero beyond p).
constexpr int YP_NT = 384;                              // yprep threads: 24 warps per SM at two blocks
__global__ void __launch_bounds__(YP_NT, 2)
yprep_kernel(const float* __restrict__ E, long ms, int N, int m, RowSet obs, ObsNoise V,
             const float* __restrict__ Yx, const float* __restrict__ Yu, int n_yx, int KH, int pp,
             float* __restrict__ Bop, float* __restrict__ Ysh, float* __restrict__ Dbuf, float* __restrict__ Bd,
             int KCD)
{
    pdl_begin();
    extern __shared__ float Ds[];                 // [32][ldd]: D transposed, [j][c]
    const int p = obs.count;
    const int i = blockIdx.x / KH, kh = blockIdx.x % KH;
    const int ldd = 32 * KCD + 1;
    if (Bd != nullptr)
        for (int e = threadIdx.x; e < 32 * (32 * KCD - pp); e += YP_NT) {
            const int jj = e / (32 * KCD - pp), c = pp + e % (32 * KCD - pp);
            Ds[jj * ldd + c] = 0.f;
        }
    char* tile = reinterpret_cast<char*>(Bop) + ((size_t)i * KH + kh) * (size_t)(2 * pp) * 128;
    // YU units of a thread per round: every load of the round issued before the
    // first is used (one round trip to memory; one round up to pp = 144)
    constexpr int YU = 3;
    const int units = pp * 8;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int base = 0; base < units; base += YP_NT * YU) {
        float4 yv[YU], y0v[YU], ybv[YU];
#pragma unroll
        for (int u = 0; u < YU; ++u) {
            const int e = base + threadIdx.x + YP_NT * u;
            const int c = e / 8, j = kh * KC + (e % 8) * 4;
            yv[u] = y0v[u] = ybv[u] = zero;
            if (e < units && c < p && j < m) {
                yv[u] = __ldg(reinterpret_cast<const float4*>(E + (long)i * ms + (long)obs.rows[c] * m + j));
                y0v[u] = __ldg(reinterpret_cast<const float4*>(E + (long)obs.rows[c] * m + j));
                if (c < p - obs.nc) {
                    const float* yb = c < n_yx ? Yx + (long)c * m : Yu + (long)(c - n_yx) * m;
                    ybv[u] = *reinterpret_cast<const float4*>(yb + j);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < YU; ++u) {
            const int e = base + threadIdx.x + YP_NT * u;
            if (e >= units) break;
            const int c = e / 8, k = e % 8;
            const int j = kh * KC + k * 4;
            float4 hi = zero, lo = zero, d = zero;
            if (c < p && j < m) {
                const float4 y = f4add(yv[u], obs_noise4(V, obs, p, i, c, j, m));
                const float4 ev = f4sub(y, y0v[u]);
                split_tf32(ev, hi, lo);
                *reinterpret_cast<float4*>(Ysh + ((long)i * p + c) * m + j) = ev;
                d = f4sub(ybv[u], y);                       // constraint rows: reference 0
                if (Dbuf != nullptr) *reinterpret_cast<float4*>(Dbuf + ((long)i * p + c) * m + j) = d;
            }
            if (Bd != nullptr) {
                Ds[(k * 4 + 0) * ldd + c] = d.x;
                Ds[(k * 4 + 1) * ldd + c] = d.y;
                Ds[(k * 4 + 2) * ldd + c] = d.z;
                Ds[(k * 4 + 3) * ldd + c] = d.w;
            }
            *reinterpret_cast<float4*>(tile + swz(c, k)) = hi;
            *reinterpret_cast<float4*>(tile + swz(pp + c, k)) = lo;
        }
    }
    if (Bd == nullptr) return;
    __syncthreads();
    const long NM = (long)N * m;
    char* bd = reinterpret_cast<char*>(Bd);
    for (int e = threadIdx.x; e < 32 * KCD * 8; e += YP_NT) {
        const int jj = e / (KCD * 8), kc = (e / 8) % KCD, q = e % 8;
        const int j = kh * KC + jj;
        if (j >= m) continue;
        const long n = (long)i * m + j;
        const float* src = Ds + jj * ldd + kc * 32 + q * 4;
        float4 hi, lo;
        split_tf32(make_float4(src[0], src[1], src[2], src[3]), hi, lo);
        const int off = (int)((n & 7) ^ q) << 4;
        *reinterpret_cast<float4*>(bd + ((size_t)(2 * kc) * NM + n) * 128 + off) = hi;
        *reinterpret_cast<float4*>(bd + ((size_t)(2 * kc + 1) * NM + n) * 128 + off) = lo;
    }
}

// a left row's source: member 0's row and the stride between members (E
// rows, shifted by member 0's value; or the observation rows e_i yprep
// wrote, already shifted by the same constant as the right-hand side, so
// that S1 of these rows is the right-hand side's sum)
struct RowSrc {
    const float* e;
    long stride;
    bool live;
    bool shift;
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
                int tmem_cols, int M, float* __restrict__ part1, float* __restrict__ part2, int* __restrict__ err)
{
    pdl_trigger();
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = tc::smem_u32(smem_raw);
    const uint32_t s0 = (raw + 1023u) & ~1023u;                     // swizzle atoms need 1024-byte alignment
    unsigned char* smem = smem_raw + (s0 - raw);
    const int R = act.count, p = obs.count;             // left rows: act rows, then obs rows, cut at M <= R + p
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
    pdl_wait();                                         // the set-up above reads no kernel's output
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
                src[u].shift = true;
            } else {
                src[u].e = Ysh + (long)(a < M ? a - R : 0) * m;
                src[u].stride = (long)p * m;
                src[u].shift = false;
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
                    v0[u] = src[u].shift ? load_unit(src[u], 0, j, m) : make_float4(0.f, 0.f, 0.f, 0.f);
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
            // two 16-column groups per TMEM wait; 16-byte stores of the row
            float* prow = part2 + ((long)sidx * M + a) * p;
            const bool vec = (p & 3) == 0;
            for (int c0 = (warp >> 2) * 16; c0 < pp; c0 += 64) {
                float v[2][16];
                const bool two = c0 + 32 < pp;       // warp-uniform
                tc::tmem_ld16(tmem + tl + c0, v[0]);
                if (two) tc::tmem_ld16(tmem + tl + c0 + 32, v[1]);
                tc::tmem_ld_wait();
                if (a < M) {
#pragma unroll
                    for (int g = 0; g < 2; ++g) {
                        const int cg = c0 + 32 * g;
                        if (g == 1 && !two) break;
#pragma unroll
                        for (int u4 = 0; u4 < 4; ++u4) {
                            const int c = cg + 4 * u4;
                            float4 x = make_float4(v[g][4 * u4], v[g][4 * u4 + 1], v[g][4 * u4 + 2], v[g][4 * u4 + 3]);
                            if (nst == 0) x = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (vec && c + 3 < p) {
                                *reinterpret_cast<float4*>(prow + c) = x;
                            } else {
                                if (c < p) prow[c] = x.x;
                                if (c + 1 < p) prow[c + 1] = x.y;
                                if (c + 2 < p) prow[c + 2] = x.z;
                                if (c + 3 < p) prow[c + 3] = x.w;
                            }
                        }
                    }
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
    } else if (warp == ST_ISSUER) {
        // ---- issuer: per stage 4 K steps of 8, three MMAs each; the whole
        // warp runs the loop (warp-uniform operands, outcomes agreed by
        // vote) and the elected lane issues
        const uint32_t id = idesc_tf32(TM, pp);
        for (int q = 0; q < nst; ++q) {
            const int s = q % S;
            const uint32_t par = (uint32_t)((q / S) & 1);
            const bool got = tc::mbar_wait_bounded(full + s, par, ST_WAIT) && tc::mbar_wait_bounded(bful + s, par, ST_WAIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicExch(err, DEV_TIMEOUT);
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
                st_mma_el(tmem, ah, bh, id, (q | ks) != 0 ? 1u : 0u);
                st_mma_el(tmem, ah, bl, id, 1u);
                st_mma_el(tmem, al, bh, id, 1u);
            }
            tc::mma_commit_elect(freeb + s);
        }
        tc::mma_commit_elect(done);
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
// one wave of at most 148 CTAs, and at least 4 members per split: fewer
// stages per CTA against more partial sums to reduce (measured at 64 x 64,
// N = 256: 4 members per split beat 6 and 3)
int stats_tc_splits(int M, int N)
{
    int s = 148 / stats_tc_rtiles(M);
    if (s > N / 4) s = N / 4;
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

void launch_yprep_tc(const float* E, long ms, int N, int m, RowSet obs, ObsNoise V, const float* Yx, const float* Yu,
                     int n_yx, float* Bop, float* Dbuf, float* Bd, cudaStream_t st)
{
    const int p = obs.count, pp = stats_tc_pp(p), KH = stats_tc_kh(m);
    const int KCD = (p + 31) / 32;
    float* Ysh = Bop + (size_t)N * KH * 2 * pp * 32;      // after the observation tiles
    const size_t ysm = Bd != nullptr ? sizeof(float) * 32 * (32 * KCD + 1) : 0;
    pdl_launch(yprep_kernel, N * KH, YP_NT, ysm, st, E, ms, N, m, obs, V, Yx, Yu, n_yx, KH, pp, Bop, Ysh, Dbuf, Bd, KCD);
}

void launch_stats_tc_rows(const float* E, long ms, int N, int m, RowSet act, RowSet obs, int M, const float* Bop,
                          float* part1, float* part2, int splits, int* err, cudaStream_t st)
{
    const int p = obs.count, pp = stats_tc_pp(p), KH = stats_tc_kh(m);
    const float* Ysh = Bop + (size_t)N * KH * 2 * pp * 32;
    const int S = st_stages(pp);
    const int cols = pp <= 32 ? 32 : pp <= 64 ? 64 : pp <= 128 ? 128 : 256;
    const size_t smem = stats_tc_smem(p);
    cudaFuncSetAttribute(stats_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pdl_launch(stats_tc_kernel, dim3(stats_tc_rtiles(M), splits), ST_NT, smem, st, E, ms, N, m, act, obs, Ysh, Bop, pp,
               KH, S, splits, cols, M, part1, part2, err);
}

void launch_stats_tc(const float* E, long ms, int N, int m, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
                     const float* Yu, int n_yx, float* Bop, float* part1, float* part2, float* Dbuf, float* Bd,
                     int splits, int* err, cudaStream_t st)
{
    launch_yprep_tc(E, ms, N, m, obs, V, Yx, Yu, n_yx, Bop, Dbuf, Bd, st);
    launch_stats_tc_rows(E, ms, N, m, act, obs, act.count + obs.count, Bop, part1, part2, splits, err, st);
}

}  // namespace oic
