// noalloc_api.cu -- oic_enks_update_static: the ensemble Kalman analysis
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a real-time control loop that
// must never reach the allocator after start-up (an allocation can block or
// fail at any time), a plug-in whose host process owns the GPU memory pool
// and forbids allocations of its own, or an embedding with a fixed memory
// map.  For them this
// entry point runs the same kernels as oic_enks_update but keeps every
// intermediate (split-K partial sums, innovations, covariances, gain, row
// tables, status word) in one file-scope device array of fixed size,
// OIC_STATIC_SCRATCH_BYTES, that the CUDA module carries.  The caller passes
// only its inputs and outputs.  The array exists once per GPU that loads the
// library and stays reserved until the process exits.
#include <cstdint>
#include <mutex>

#include "oic_internal.cuh"

namespace {

constexpr size_t SCRATCH_BYTES = OIC_STATIC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_oic_scratch[SCRATCH_BYTES];

std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
oic_status scratch_for_current_device(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return OIC_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_oic_scratch) != cudaSuccess || p == nullptr) return OIC_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return OIC_OK;
}

// True when p is device memory of the current device (or managed memory,
// which the current device can reach).  A pointer into another GPU's memory
// or into pageable host memory is refused before anything is launched.
bool on_current_device(const void* p, int dev)
{
    cudaPointerAttributes a = {};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" oic_status oic_enks_update_static(int N, int R, int m, int p, const int* obs_rows, float* E,
                                             const float* V, const float* Ybar, void* cuda_stream)
{
    using namespace oic;
    if (!obs_rows || !E || !V || !Ybar) return OIC_EINVAL;
    if (N < 2 || R < 1 || m < 4 || m > 128 || m % 4 != 0 || p < 1 || p > 144) return OIC_EINVAL;
    if ((reinterpret_cast<uintptr_t>(E) & 15u) || (reinterpret_cast<uintptr_t>(V) & 15u)) return OIC_EINVAL;
    if ((long)N * m > (1L << 28)) return OIC_EINVAL;
    for (int c = 0; c < p; ++c)
        if (obs_rows[c] < 0 || obs_rows[c] >= R) return OIC_EINVAL;

    // carve the scratch exactly as the handle's workspace is carved
    const int M = R + p;
    const int splits = stats_splits(R, p, N);
    const size_t off_part1 = 0;
    const size_t off_part2 = off_part1 + up256(sizeof(float) * (size_t)splits * M * m);
    const size_t off_S1 = off_part2 + up256(sizeof(float) * (size_t)splits * M * p);
    const size_t off_D = off_S1 + up256(sizeof(float) * (size_t)M * m);
    const size_t off_C = off_D + up256(sizeof(float) * (size_t)N * p * m);
    const size_t off_K = off_C + up256(sizeof(double) * (size_t)M * p);
    const size_t off_rows = off_K + up256(sizeof(float) * (size_t)p * R);
    const size_t off_status = off_rows + up256(sizeof(int) * (size_t)(R + p));
    const size_t need = off_status + 256;
    if (need > SCRATCH_BYTES) return OIC_ENOMEM;   // sizes beyond the static scratch

    unsigned char* base = nullptr;
    const oic_status st = scratch_for_current_device(&base);
    if (st != OIC_OK) return st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OIC_ECUDA;
    if (!on_current_device(E, dev) || !on_current_device(V, dev) || !on_current_device(Ybar, dev))
        return OIC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // row tables: active rows 0 .. R-1, then the observed rows (copied from
    // host memory that may be released as soon as this call returns)
    int* rows = reinterpret_cast<int*>(base + off_rows);
    int* status = reinterpret_cast<int*>(base + off_status);
    int host_rows[1024];
    int done = 0;
    while (done < R + p) {
        const int cnt = (R + p - done) < 1024 ? (R + p - done) : 1024;
        for (int k = 0; k < cnt; ++k) {
            const int r = done + k;
            host_rows[k] = r < R ? r : obs_rows[r - R];
        }
        if (cudaMemcpyAsync(rows + done, host_rows, sizeof(int) * cnt, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return OIC_ECUDA;
        done += cnt;
    }
    // the status word must start at zero; every other region is written in
    // full before it is read
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return OIC_ECUDA;

    float* part1 = reinterpret_cast<float*>(base + off_part1);
    float* part2 = reinterpret_cast<float*>(base + off_part2);
    float* S1 = reinterpret_cast<float*>(base + off_S1);
    float* D = reinterpret_cast<float*>(base + off_D);
    double* C = reinterpret_cast<double*>(base + off_C);
    float* Kt = reinterpret_cast<float*>(base + off_K);
    RowSet act{rows, R};
    RowSet obs{rows + R, p};
    const ObsNoise Vn = obs_noise_buf(V, V, p);
    const long ms = (long)R * m;
    launch_stats(E, ms, N, m, act, obs, Vn, Ybar, Ybar, p, part1, part2, D, splits, s);
    launch_s1_reduce(part1, splits, M, m, S1, s);
    launch_cov_finalize(part2, S1, splits, R, p, m, N, C, s);
    launch_gain(C, R, p, Kt, status, s);
    launch_update(E, ms, N, m, act, Kt, p, D, s);
    if (cudaGetLastError() != cudaSuccess) return OIC_ECUDA;

    int dev_status = 0;
    if (cudaMemcpyAsync(&dev_status, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return OIC_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return OIC_ECUDA;
    return dev_status == DEV_NOTSPD ? OIC_ENOTSPD : OIC_OK;
}
