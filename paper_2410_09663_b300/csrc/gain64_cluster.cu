// gain64_cluster.cu -- the mixed-precision mode's FP64 gain,
// K = Sigma^XY (Sigma^Y)^-1 by the Cholesky factorisation Sigma^Y = L L^T
// and two substitutions per gain row (Eq. of the sample-wise ensemble
// Kalman update; the factorisation as in the Appendix).
//
// B300's FP64 pipe does about 2 FMA/clk/SM, so a one-CTA factorisation of
// p = 144 (p^3/3 = 1e6 FMA) costs at least 250 us.  Here it runs on a cluster
// of 8 CTAs (8 SMs):
//   - rows are distributed block-cyclically in panels of 8: panel B (rows
//     8B .. 8B+7) lives in the shared memory of CTA B mod 8;
//   - per panel, the owner eliminates its 8 pivots (right-looking, upper
//     form Sigma^Y = U^T U with U = L^T), scales the rows to U and releases
//     them with one remote mbarrier arrive (release, cluster scope) on every
//     CTA of the cluster;
//   - every CTA waits for that barrier (acquire, cluster scope, bounded),
//     copies the panel out of the owner's shared memory (distributed shared
//     memory) and applies the rank-8 update to its own later rows, the next
//     panel's rows first: their owner then eliminates and releases the next
//     panel before it updates the rest (look-ahead), so a panel's release
//     waits for one panel's update of 8 rows, not of every later row;
//   - a pivot <= 0 ("not positive definite") is published with the panel, so
//     every CTA leaves the loop after the same panel.
// Each panel barrier is used once (parity 0), so no barrier ever has two
// phases outstanding.  The cluster barrier at the end keeps every CTA's
// shared memory alive until the others have read it.  Then solve64_kernel
// gives each gain row one warp (L staged in shared memory; column-form FP64
// forward and back substitution).
#include "oic_internal.cuh"
#include "tc_sm103.cuh"

namespace oic {
namespace {

constexpr int CL = 8;                                   // CTAs per cluster
constexpr int PB = 8;                                   // rows per panel
constexpr int C64_T = 256;
constexpr int C64_PMAX = 160;                           // largest p
constexpr int C64_NB = C64_PMAX / PB;                   // panels at most
constexpr int C64_OWN = (C64_NB + CL - 1) / CL;         // panels per CTA at most
constexpr long long C64_WAIT = 4000000000LL;

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(tc::smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ double cl_ld(uint32_t addr)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ int cl_ld_s32(uint32_t addr)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cl_arrive(uint32_t mbar_cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar_cluster_addr) : "memory");
}
__device__ __forceinline__ bool cl_wait(uint64_t* mbar, uint32_t parity, long long max_cycles)
{
    const long long t0 = clock64();
    unsigned ns = 0;                                    // sleep between polls, 8 ns doubling to 64 ns
    for (;;) {
        if (ns) __nanosleep(ns);
        ns = ns == 0 ? 8 : ns < 64 ? 2 * ns : 64;
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(tc::smem_u32(mbar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > max_cycles) return false;
    }
}
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 1/sqrt(x) in FP64: an FP32 seed refined by two Newton steps for 1/y^2 = x
// (each step squares the relative error: 2^-23 -> 2^-46 -> FP64 rounding)
__device__ __forceinline__ double rsqrt64(double x)
{
    const float xf = (float)x;
    if (!(xf > 0.f) || xf > 1e37f) return 1.0 / sqrt(x);
    double y = (double)rsqrtf(xf);
    const double hx = 0.5 * x;
    y = y * fma(-hx, y * y, 1.5);
    y = y * fma(-hx, y * y, 1.5);
    return y;
}

__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(C64_T, 1)
chol64c_kernel(const double* __restrict__ C, int R, int p, double* __restrict__ Lg, int* __restrict__ status,
               int* __restrict__ bad_out)
{
    pdl_begin();
    __shared__ __align__(16) double own[C64_OWN][PB][C64_PMAX];    // this CTA's panels (rows of A, then of U)
    __shared__ __align__(16) double pan[PB][C64_PMAX];             // the current panel (U rows)
    __shared__ double rsv[PB], ips[PB];                          // 1 / U[g][g], 1 / pivot
    __shared__ __align__(8) uint64_t rdy[C64_NB];
    __shared__ int bad_here, bad_seen, timeout;
    const int tid = threadIdx.x, w = tid / 32, lane = tid % 32;
    const uint32_t rank = cl_rank();
    const int pp = (p + PB - 1) / PB * PB, NB = pp / PB;
    const double* Cyy = C + (long)R * p;
    for (int sl = 0; sl < C64_OWN; ++sl) {
        const int B = (int)rank + CL * sl;
        if (B >= NB) break;
        for (int e = tid; e < PB * pp; e += C64_T) {
            const int d = e / pp, c = e % pp, g = PB * B + d;
            own[sl][d][c] = (g < p && c < p) ? Cyy[(long)g * p + c] : 0.0;
        }
    }
    if (tid == 0) {
        for (int B = 0; B < NB; ++B) tc::mbar_init(rdy + B, 1);
        bad_here = 0;
        bad_seen = 0;
        timeout = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    cl_sync();                                          // every barrier initialised before any remote arrive

    // 1 / sqrt and 1 / pivot d of the panel at column c0, by warp 0 alone (the
    // pivot chain is a series of dependent FP64 operations of ~64 cycles each,
    // whatever the number of active lanes; computed by every warp, they also
    // queued behind each other on the FP64 pipe)
    auto pivot = [&](double (*A)[C64_PMAX], int c0, int d) {
        const int g = c0 + d;
        const double piv = A[d][g];
        const double r = (g < p && piv > 0.0) ? rsqrt64(piv) : 0.0;
        if (lane == 0) {
            if (g < p && !(piv > 0.0)) bad_here = 1;
            rsv[d] = r;
            ips[d] = r * r;
            if (g < p) Lg[(long)p * p + g] = r;                 // 1 / L_gg, for the substitutions
        }
    };
    // the owner eliminates panel B's pivots (right-looking, rows in own[B / CL]),
    // scales the rows to U and releases the panel to every CTA
    auto eliminate = [&](int B) {
        double (*A)[C64_PMAX] = own[B / CL];
        const int c0 = PB * B;
        if (w == 0) pivot(A, c0, 0);
        __syncthreads();
        for (int d = 0; d < PB; ++d) {
            // rows e > d of the panel, columns c >= c0 + e: warp w takes row d + 1 + w;
            // warp 0, whose row holds the next pivot, then computes its reciprocals
            const int e = d + 1 + w;
            if (e < PB) {
                const double f = A[d][c0 + e] * ips[d];
                for (int c = c0 + e + lane; c < pp; c += 32) A[e][c] = fma(-f, A[d][c], A[e][c]);
                if (w == 0) {
                    __syncwarp();
                    pivot(A, c0, d + 1);
                }
            }
            __syncthreads();
        }
        for (int x = tid; x < PB * pp; x += C64_T) {
            const int d = x / pp, c = x % pp;
            if (c >= c0 + d) A[d][c] *= rsv[d];
        }
        __syncthreads();
        // one remote arrive per CTA of the cluster, each from its own lane (issued
        // one after another by one thread they took ~1.7 us)
        if (tid < CL) cl_arrive(cl_map(rdy + B, (uint32_t)tid));
    };
    // rank-8 update of panel B2's rows (this CTA's), columns c >= row, by the panel in pan
    auto update = [&](int B2) {
        double (*A)[C64_PMAX] = own[B2 / CL];
        for (int d2 = w; d2 < PB; d2 += C64_T / 32) {
            const int g = PB * B2 + d2;
            double pi[PB];
#pragma unroll
            for (int k = 0; k < PB; ++k) pi[k] = pan[k][g];
            for (int c = g + lane; c < pp; c += 32) {
                double v = A[d2][c];
#pragma unroll
                for (int k = 0; k < PB; ++k) v = fma(-pi[k], pan[k][c], v);
                A[d2][c] = v;
            }
        }
    };
    if (rank == 0) eliminate(0);
    for (int B = 0; B < NB; ++B) {
        const uint32_t o = (uint32_t)(B % CL);
        const int sl = B / CL, c0 = PB * B;
        // ---- everyone: wait for the panel, copy it, check the owner's pivots
        if (!cl_wait(rdy + B, 0u, C64_WAIT)) timeout = 1;
        __syncthreads();
        if (timeout) break;
        for (int x = tid; x < PB * (pp - c0); x += C64_T) {
            const int d = x / (pp - c0), c = c0 + x % (pp - c0);
            pan[d][c] = cl_ld(cl_map(&own[sl][d][c], o));
        }
        if (tid == 0) bad_seen = cl_ld_s32(cl_map(&bad_here, o));
        __syncthreads();
        if (bad_seen) break;
        // ---- look-ahead: the next panel's owner updates and releases it first
        const int Bn = B + 1;
        const bool ahead = Bn < NB && (int)rank == Bn % CL;
        if (ahead) {
            update(Bn);
            __syncthreads();
            eliminate(Bn);
        }
        // ---- then this CTA's other rows in later panels
        for (int sl2 = 0; sl2 < C64_OWN; ++sl2) {
            const int B2 = (int)rank + CL * sl2;
            if (B2 <= B || B2 >= NB || (ahead && B2 == Bn)) continue;
            update(B2);
        }
        __syncthreads();
    }
    __syncthreads();
    cl_sync();                                          // nobody reads another CTA's shared memory after this
    if (timeout && tid == 0) atomicExch(status, DEV_TIMEOUT);
    if (bad_seen || timeout) {
        if (rank == 0 && tid == 0) {
            if (bad_seen) atomicExch(status, DEV_NOTSPD);
            *bad_out = 1;
        }
        return;
    }
    if (rank == 0 && tid == 0) *bad_out = 0;
    // L[i][g] = U[g][i] for i >= g, zero above the diagonal (a panel's 8
    // columns of a row next to each other: 64-byte segments)
    for (int sl = 0; sl < C64_OWN; ++sl) {
        const int B = (int)rank + CL * sl;
        if (B >= NB) break;
        for (int x = tid; x < PB * p; x += C64_T) {
            const int d = x % PB, i = x / PB, g = PB * B + d;
            if (g < p) Lg[(long)i * p + g] = i >= g ? own[sl][d][i] : 0.0;
        }
    }
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(dst)), "l"(src) : "memory");
}

// One warp per gain row a; L staged in shared memory with an odd leading
// dimension (column reads of the forward pass and row reads of the backward
// pass are both conflict-free); lane t holds z_i for i = t + 32 q.
constexpr int S64_W = 4;                                // warps (gain rows) per CTA
constexpr int S64_Q = 5;                                // p <= 160

// The forward substitution's pivots j in slot QJ (j = 32 QJ + lj): lane i
// of slot q holds z_{32 q + i}.
template <int QJ>
__device__ __forceinline__ void fwd_slot(double (&z)[S64_Q], const double* __restrict__ Ls,
                                         const double* __restrict__ rinv, int ld, int p, int lane)
{
    static_assert(QJ < S64_Q, "slot");
    const int j0 = 32 * QJ, j1 = p < j0 + 32 ? p : j0 + 32;
    for (int j = j0; j < j1; ++j) {
        const int lj = j - j0;
        const double zj = __shfl_sync(0xffffffffu, z[QJ], lj) * rinv[j];
        if (lane == lj) z[QJ] = zj;
        else if (lane > lj && j0 + lane < p) z[QJ] = fma(-Ls[(j0 + lane) * ld + j], zj, z[QJ]);
#pragma unroll
        for (int q = QJ + 1; q < S64_Q; ++q) {
            const int i = lane + 32 * q;
            if (32 * q < p && i < p) z[q] = fma(-Ls[i * ld + j], zj, z[q]);
        }
    }
}
// The backward substitution's pivots j in slot QJ, from the top of the slot down.
template <int QJ>
__device__ __forceinline__ void bwd_slot(double (&z)[S64_Q], const double* __restrict__ Ls,
                                         const double* __restrict__ rinv, int ld, int p, int lane)
{
    static_assert(QJ < S64_Q, "slot");
    const int j0 = 32 * QJ, j1 = p < j0 + 32 ? p : j0 + 32;
    for (int j = j1 - 1; j >= j0; --j) {
        const int lj = j - j0;
        const double kj = __shfl_sync(0xffffffffu, z[QJ], lj) * rinv[j];
        if (lane == lj) z[QJ] = kj;
        else if (lane < lj) z[QJ] = fma(-Ls[j * ld + j0 + lane], kj, z[QJ]);
#pragma unroll
        for (int q = 0; q < QJ; ++q) z[q] = fma(-Ls[j * ld + lane + 32 * q], kj, z[q]);
    }
}

__global__ void __launch_bounds__(32 * S64_W)
solve64s_kernel(const double* __restrict__ C, int R, int p, const double* __restrict__ Lg,
                const int* __restrict__ bad_in, float* __restrict__ Kt)
{
    pdl_begin();
    extern __shared__ double Ls[];                      // [p][p | 1], then 1 / L_ii
    const int ld = p | 1;
    double* rinv = Ls + (size_t)p * ld;
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int a = blockIdx.x * S64_W + w;
    if (*bad_in) {
        if (a < R)
            for (int i = lane; i < p; i += 32) Kt[(long)i * R + a] = 0.f;
        return;
    }
    // the lower triangle of L and 1 / L_ii (written by the factorisation) by
    // asynchronous 8-byte copies, all in flight at once (one round trip)
    for (int i = w; i < p; i += S64_W)
        for (int k = lane; k <= i; k += 32) cp_async8(Ls + i * ld + k, Lg + (long)i * p + k);
    for (int i = threadIdx.x; i < p; i += 32 * S64_W) cp_async8(rinv + i, Lg + (long)p * p + i);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (a >= R) return;
    double z[S64_Q];
#pragma unroll
    for (int q = 0; q < S64_Q; ++q) {
        const int i = lane + 32 * q;
        z[q] = i < p ? C[(long)a * p + i] : 0.0;
    }
    // forward: z_j /= L_jj, then z_i -= L_ij z_j for i > j (column j of L);
    // back: k_j = z_j / L_jj, then z_i -= L_ji k_j for i < j (row j of L).
    // The pivots of slot QJ (j = 32 QJ .. 32 QJ + 31) are taken together, QJ a
    // compile-time constant: z_j comes straight from slot QJ and the slots
    // wholly past the pivot are known, so each step issues only its FP64
    // multiply and the FMAs of the live slots (B300's FP64 pipe is the limit).
    fwd_slot<0>(z, Ls, rinv, ld, p, lane);
    fwd_slot<1>(z, Ls, rinv, ld, p, lane);
    fwd_slot<2>(z, Ls, rinv, ld, p, lane);
    fwd_slot<3>(z, Ls, rinv, ld, p, lane);
    fwd_slot<4>(z, Ls, rinv, ld, p, lane);
    bwd_slot<4>(z, Ls, rinv, ld, p, lane);
    bwd_slot<3>(z, Ls, rinv, ld, p, lane);
    bwd_slot<2>(z, Ls, rinv, ld, p, lane);
    bwd_slot<1>(z, Ls, rinv, ld, p, lane);
    bwd_slot<0>(z, Ls, rinv, ld, p, lane);
#pragma unroll
    for (int q = 0; q < S64_Q; ++q) {
        const int i = lane + 32 * q;
        if (i < p) Kt[(long)i * R + a] = (float)z[q];
    }
}

}  // namespace

int gain64_max_p() { return C64_PMAX; }

void launch_chol64(const double* C, int R, int p, double* L, int* bad, int* status, cudaStream_t st)
{
    pdl_launch(chol64c_kernel, CL, C64_T, 0, st, C, R, p, L, status, bad);
}

void launch_solve64(const double* C, int R, int p, const double* L, const int* bad, float* Kt, cudaStream_t st)
{
    const size_t smem = sizeof(double) * ((size_t)p * (p | 1) + p);
    static DeviceOnce attr_set;
    attr_set.run([] {
        return cudaFuncSetAttribute(solve64s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(double) * ((size_t)C64_PMAX * (C64_PMAX | 1) + C64_PMAX))) ==
               cudaSuccess;
    });
    pdl_launch(solve64s_kernel, (R + S64_W - 1) / S64_W, 32 * S64_W, smem, st, C, R, p, L, bad, Kt);
}

void launch_gain64(const double* C, int R, int p, double* L, int* bad, float* Kt, int* status, cudaStream_t st)
{
    launch_chol64(C, R, p, L, bad, status, st);
    launch_solve64(C, R, p, L, bad, Kt, st);
}

}  // namespace oic
