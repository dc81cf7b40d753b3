// update_tc.cu -- the member update of the analysis (Eq. of the sample-wise
// ensemble Kalman update): X^i[a] += sum_c K[a][c] D^i[c] for every active
// row a and every member i, as one GEMM on the tcgen05 tensor cores:
//
//   E[rows a][columns n = (i, j)] += sum_c K[a][c] Bd[n][c]
//
// computed transposed, acc[n][a] = sum_c Bd[n][c] K[a][c]: M = a group of
// 128 ensemble columns, N = a tile of 128 of the R active rows, K = p
// (chunks of 32).  A tensor-memory lane is then one ensemble column, so for
// each active row the 32 lanes of a drain warp add into 32 consecutive
// values of the ensemble row: one 128-byte run per warp access.  FP32
// accuracy from TF32 operands split x = hi + lo, three products per K step
// in two MMAs: D_hi [K_hi; K_lo] (N = 256: the gain tile's hi and lo rows
// are contiguous) into accumulator columns [0, 256), then D_lo K_hi into
// columns [128, 256); the result is columns a + (128 + a).  Two MMA issues
// per K step instead of three, with the same tensor-pipe cycles (a single
// issuing thread needs about as long to issue an N = 128 MMA as the tensor
// core to run it).  Operands, both 128-byte-swizzled K-major tiles:
//   Aop [row tile][kc][hi | lo][128 rows][32 values]   from the gain (kprep)
//   Bd  [kc][hi | lo][N m rows][32 values]             from yprep_kernel
// A persistent grid walks work items (column group, row tile), row tile
// fastest so that consecutive items of a CTA reuse the same Bd rows from L2.
// Per item a loader bulk-copies one stage per K chunk (A hi / lo and
// B hi / lo, 64 KB) into a 3-stage ring, one warp (an elected lane) issues the MMAs into
// one of two tensor-memory accumulators, and sixteen drain warps add the
// finished accumulator into the ensemble (one lane per column, 16 rows per
// tensor-memory load) while the next item accumulates into the other one.
#include "oic_internal.cuh"
#include "tc_sm103.cuh"
#include "tc_tf32.cuh"

namespace oic {
namespace {

using namespace tf32;

constexpr int UT_M = 128;                               // rows per tile
constexpr int UT_N = 128;                               // columns per item
constexpr int UT_KC = 32;                               // K values per stage
constexpr int UT_PART = UT_M * 128;                     // one operand part (hi or lo), bytes
constexpr int UT_ACC = 2 * UT_N;                        // accumulator columns: [hi hi | hi lo + lo hi]
constexpr int UT_STAGE = 4 * UT_PART;                   // A hi, A lo, B hi, B lo
constexpr int UT_S = 3;                                 // ring stages
constexpr int UT_DW = 16;                               // drain warps: four per tensor-memory lane quarter
constexpr int UT_NT = (UT_DW + 2) * 32;                 // drain warps, loader, issuer
constexpr int UT_LOADER = UT_DW, UT_ISSUER = UT_DW + 1;
constexpr int UT_DR = UT_M * 4 / UT_DW;                 // active rows a drain warp adds
constexpr long long UT_WAIT = 4000000000LL;

// Kt [p][R] (K transposed) -> Aop tiles; one thread per (row tile, kc, row,
// 16-byte chunk), rows of a warp consecutive (coalesced reads of Kt).
__global__ void kprep_kernel(const float* __restrict__ Kt, int R, int p, int rtiles, int KCH,
                             float* __restrict__ Aop)
{
    pdl_begin();
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)rtiles * KCH * 8 * UT_M) return;
    const int r = (int)(e % UT_M);
    const int q = (int)((e / UT_M) % 8);
    const int kc = (int)((e / (UT_M * 8)) % KCH);
    const int rt = (int)(e / ((long)UT_M * 8 * KCH));
    const int a = rt * UT_M + r, c0 = kc * UT_KC + q * 4;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = (a < R && c0 + u < p) ? Kt[(long)(c0 + u) * R + a] : 0.f;
    float4 hi, lo;
    split_tf32(make_float4(v[0], v[1], v[2], v[3]), hi, lo);
    char* t = reinterpret_cast<char*>(Aop) + ((size_t)rt * KCH + kc) * 2 * UT_PART;
    *reinterpret_cast<float4*>(t + swz(r, q)) = hi;
    *reinterpret_cast<float4*>(t + UT_PART + swz(r, q)) = lo;
}

__global__ void __launch_bounds__(UT_NT, 1)
update_tc_kernel(float* __restrict__ E, long ms, int m, RowSet act, const float* __restrict__ Aop,
                 const float* __restrict__ Bd, long NM, int KCH, int rtiles, int items, int* __restrict__ err)
{
    pdl_trigger();
    extern __shared__ unsigned char usm_raw[];
    const uint32_t raw = tc::smem_u32(usm_raw);
    const uint32_t s0 = (raw + 1023u) & ~1023u;
    unsigned char* smem = usm_raw + (s0 - raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + UT_S * UT_STAGE);
    uint64_t* freeb = full + UT_S;
    uint64_t* accf = freeb + UT_S;                          // [2] accumulator ready
    uint64_t* accd = accf + 2;                              // [2] accumulator drained (4 warps)
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accd + 2);
    int* row_off = reinterpret_cast<int*>(smem + UT_S * UT_STAGE + 128);   // [drain warp][UT_DR]
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int R = act.count;
    const int t0 = (int)((long)blockIdx.x * items / gridDim.x);
    const int t1 = (int)((long)(blockIdx.x + 1) * items / gridDim.x);
    if (tid == 0) {
        for (int s = 0; s < UT_S; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(freeb + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(accf + b, 1);
            tc::mbar_init(accd + b, UT_DW);
        }
        tc::fence_mbar_init();
    }
    if (warp == UT_LOADER) {
        tc::tmem_alloc(tmem_holder, 2 * UT_ACC);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    pdl_wait();                                         // the set-up above reads no kernel's output
    const int nst = (t1 - t0) * KCH;

    if (warp == UT_LOADER && lane == 0) {
        int q = 0;
        for (; q < nst; ++q) {
            const int s = q % UT_S;
            if (q >= UT_S && !tc::mbar_wait_bounded(freeb + s, (uint32_t)((q / UT_S - 1) & 1), UT_WAIT)) {
                atomicExch(err, DEV_TIMEOUT);
                break;
            }
            const int t = t0 + q / KCH, kc = q % KCH;
            const int g = t / rtiles, rt = t % rtiles;
            const long n0 = (long)g * UT_N;
            const int rows = NM - n0 < UT_N ? (int)(NM - n0) : UT_N;
            const uint32_t dst = s0 + s * UT_STAGE;
            const char* a = reinterpret_cast<const char*>(Aop) + ((size_t)rt * KCH + kc) * 2 * UT_PART;
            const char* b = reinterpret_cast<const char*>(Bd) + ((size_t)(2 * kc) * NM + n0) * 128;
            st_expect_tx(full + s, 2 * UT_PART + 2 * rows * 128);
            st_bulk(dst, a, 2 * UT_PART, full + s);
            st_bulk(dst + 2 * UT_PART, b, rows * 128, full + s);
            st_bulk(dst + 3 * UT_PART, b + (size_t)NM * 128, rows * 128, full + s);
        }
        for (int r = q - UT_S < 0 ? 0 : q - UT_S; r < q; ++r)
            tc::mbar_wait_bounded(full + r % UT_S, (uint32_t)((r / UT_S) & 1), UT_WAIT);
    } else if (warp == UT_ISSUER) {
        // the whole warp runs the issue loop (warp-uniform operands, outcomes
        // agreed by vote); the elected lane issues each MMA and commit
        const uint32_t id2 = idesc_tf32(UT_M, 2 * UT_N), id1 = idesc_tf32(UT_M, UT_N);
        bool ok = true;
        for (int u = 0; u < t1 - t0 && ok; ++u) {
            const int buf = u & 1;
            const uint32_t acc = tmem + buf * UT_ACC;
            if (u >= 2 &&
                !__all_sync(0xffffffffu, tc::mbar_wait_bounded(accd + buf, (uint32_t)((u / 2 - 1) & 1), UT_WAIT))) {
                if (lane == 0) atomicExch(err, DEV_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            for (int kc = 0; kc < KCH; ++kc) {
                const int q = u * KCH + kc, s = q % UT_S;
                if (!__all_sync(0xffffffffu, tc::mbar_wait_bounded(full + s, (uint32_t)((q / UT_S) & 1), UT_WAIT))) {
                    if (lane == 0) atomicExch(err, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t base = s0 + s * UT_STAGE;
#pragma unroll
                for (int ks = 0; ks < UT_KC / 8; ++ks) {
                    const uint32_t k2 = sw_desc(base + ks * 32);                  // gain rows hi | lo (N = 256)
                    const uint32_t dh = sw_desc(base + 2 * UT_PART + ks * 32);    // ensemble columns (M)
                    const uint32_t dl = sw_desc(base + 3 * UT_PART + ks * 32);
                    st_mma_el(acc, dh, k2, id2, (kc | ks) != 0 ? 1u : 0u);
                    st_mma_el(acc + UT_N, dl, k2, id1, 1u);
                }
                tc::mma_commit_elect(freeb + s);
            }
            tc::mma_commit_elect(accf + buf);
        }
    } else if (warp < UT_DW) {
        // drain: lane = ensemble column n (tensor-memory lane 32 (warp % 4) +
        // lane), accumulator column = active row a of the tile; the warps of
        // one lane quarter take consecutive runs of UT_DR of the tile's rows.
        // The item's ensemble values are loaded before the accumulator is
        // waited for (they overlap the MMAs), then added 16 rows per
        // tensor-memory load; for each row the warp's loads and stores are one
        // run of 32 consecutive columns (two runs where it crosses a member's
        // last column).  Sixteen warps keep a whole item's loads in flight.
        for (int u = 0; u < t1 - t0; ++u) {
            const int buf = u & 1;
            const int t = t0 + u, g = t / rtiles, rt = t % rtiles;
            const int quarter = warp & 3, a0 = (warp >> 2) * UT_DR;
            const long n = (long)g * UT_N + 32 * quarter + lane;
            const bool live = n < NM;
            const long i = live ? n / m : 0;
            float* const col = E + i * ms + (live ? n - i * m : 0);
            const int nt = R - rt * UT_M < UT_M ? R - rt * UT_M : UT_M;       // rows of this tile, >= 1
            const int na = nt - a0;                                          // of this warp (may be <= 0)
            // the warp's row offsets, its own copy (read back as broadcasts)
            int* const off = row_off + warp * UT_DR;
            __syncwarp();                                   // the previous item's reads are done
            for (int k = lane; k < UT_DR; k += 32) off[k] = k < na ? act.rows[rt * UT_M + a0 + k] * m : 0;
            __syncwarp();
            float ev[UT_DR];
#pragma unroll
            for (int a = 0; a < UT_DR; ++a) ev[a] = (a < na && live) ? col[off[a]] : 0.f;
            bool ok = true;
            if (lane == 0) ok = tc::mbar_wait_bounded(accf + buf, (uint32_t)((u / 2) & 1), UT_WAIT);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(err, DEV_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            const uint32_t tl = tmem + buf * UT_ACC + a0 + ((uint32_t)(32 * quarter) << 16);
#pragma unroll
            for (int c = 0; c < UT_DR / 16; ++c) {
                if (16 * c >= na) break;                                     // warp-uniform
                float v[16], w[16];
                tc::tmem_ld16(tl + 16 * c, v);
                tc::tmem_ld16(tl + UT_N + 16 * c, w);
                tc::tmem_ld_wait();
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int a = 16 * c + r;
                    if (a < na && live) col[off[a]] = ev[a] + (v[r] + w[r]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(accd + buf);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == UT_LOADER) tc::tmem_dealloc(tmem, 2 * UT_ACC);
}

size_t update_tc_smem() { return 1024 + (size_t)UT_S * UT_STAGE + 128 + UT_DW * UT_DR * sizeof(int); }

}  // namespace

bool update_tc_supported(int m, int p) { return m % 16 == 0 && p >= 1 && update_tc_smem() <= 232448; }
int update_tc_kch(int p) { return (p + UT_KC - 1) / UT_KC; }
size_t update_tc_abytes(int Rmax, int p) { return (size_t)((Rmax + UT_M - 1) / UT_M) * update_tc_kch(p) * 2 * UT_PART; }
size_t update_tc_bbytes(int N, int m, int p) { return (size_t)update_tc_kch(p) * 2 * N * m * 128; }

void launch_update_tc(float* E, long ms, int N, int m, RowSet act, const float* Kt, int p, float* Aop, int max_ctas,
                      const float* Bd, int* err, cudaStream_t st, bool prep_gain)
{
    const int R = act.count, rtiles = (R + UT_M - 1) / UT_M, KCH = update_tc_kch(p);
    const long prep = (long)rtiles * KCH * 8 * UT_M;
    if (prep_gain) pdl_launch(kprep_kernel, (unsigned)((prep + 255) / 256), 256, 0, st, Kt, R, p, rtiles, KCH, Aop);
    const long NM = (long)N * m;
    const int items = (int)((NM + UT_N - 1) / UT_N) * rtiles;
    const int cap = max_ctas > 0 ? max_ctas : 148;
    const int grid = items < cap ? items : cap;
    const size_t smem = update_tc_smem();
    static DeviceOnce attr_set;
    attr_set.run([smem] {
        return cudaFuncSetAttribute(update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
               cudaSuccess;
    });
    pdl_launch(update_tc_kernel, grid, UT_NT, smem, st, E, ms, m, act, Aop, Bd, NM, KCH, rtiles, items, err);
}

}  // namespace oic
