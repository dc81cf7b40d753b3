// oic_api.cu -- the C ABI of liboic.so (declared in include/oic.h): handle,
// workspace layout, and the host-side orchestration of Algorithm 1
// (Kalman-MPC) over the kernels of cnn_kernels.cu, enks_kernels.cu and
// noise_kernels.cu.  The library never allocates device memory: every buffer
// below is carved out of the caller's workspace at oic_bind.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "oic_internal.cuh"

using namespace oic;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::atomic<unsigned long long> g_launches{0};

struct Profiler {
    bool on = false;
    unsigned mask = 0;
    int max = 0, used = 0;
    int every = 1, phase = 0;              // bracket launch i of a stage in a solve when i % every == phase
    std::vector<cudaEvent_t> ev;
    std::vector<int> stage;
};

// One control step captured as a CUDA graph (Philox noise mode: every input
// sits at a fixed workspace address and the solve index is on the device).
// The profiled variant carries an event-record node before and after each
// launch of the profiled stages; before every replay those nodes are pointed
// at fresh events of the profiler, so stage times come from the replays.
struct StepGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    unsigned mask = 0;
    int every = 1, phase = 0;              // the profiler's sampling at capture
    unsigned long long launches = 0;
    std::vector<cudaEvent_t> cap_ev;       // events named at capture, pairs
    std::vector<cudaGraphNode_t> node;     // their record nodes, same order
    std::vector<int> stage;                // stage of each pair
    bool failed = false;
    void reset()
    {
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        for (cudaEvent_t e : cap_ev) cudaEventDestroy(e);
        x = nullptr;
        g = nullptr;
        cap_ev.clear();
        node.clear();
        stage.clear();
        launches = 0;
        mask = 0;
        failed = false;
    }
};

struct Layout {
    size_t w, b, B, wtc, wfused, w16, b16, act16_in, E, act0, act1, part1, part2, S1, S1T, D, C, K, L64, tB, tAop, tBd, ctr, rowtab, status, selftest;
    size_t cG, ccols, ch;
    size_t plantX, plantU, plantTmp;
    size_t xk, uprev, xref, uref, noise, uhat, xhat, uapp, xnext;
    size_t cyy32;                     // the FP32 gain's copy of Sigma^Y (FP32 mode)
    size_t total;
};

}  // namespace

struct oic_handle {
    oic_config cfg;
    std::vector<float> w, b, B;
    int L = 0, q = 0, p = 0, R_mem = 0, R_act_max = 0, Cmax = 2;
    int Ubase = 0, splits_max = 1, n_sm = 148;
    std::vector<size_t> wtc_off;      // per layer: offset of packed tensor-core weights (or SIZE_MAX)
    size_t noise_n = 0;
    Layout lay{};
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t st = nullptr;
    bool bound = false, plant_ready = false, fused = false, bf16 = false;
    std::vector<size_t> w16_off, b16_off;   // mixed-precision CNN: packed layer tiles, padded biases
    // constraint rows: G packed over the nk non-zero columns of [Gx Gu]
    int nc = 0, nk = 0, zrow = 0;
    std::vector<float> cG, ch;
    std::vector<int> ccols;
    float c_alpha = 1.f, c_beta = 1.f, c_sigma = 0.f;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<int> obs_host;
    Profiler prof;
    oic_plan plan{};                          // scheduling choices (0 = the built-in rule)
    int stage_seen[OIC_NUM_STAGES] = {};      // launches of each stage in the current solve (and its plant step)
    StepGraph sg[2];                          // [0] plain, [1] with profiling event nodes
    StepGraph* capturing = nullptr;

    template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
    bool full() const { return cfg.keep_full_history != 0; }
    int xrow(int s) const { return full() ? s * cfg.n : (s % 2) * cfg.n; }
    int urow(int s) const { return Ubase + s * cfg.l; }
    int R_of(int s) const {
        return full() ? s * cfg.n + (s + 1) * cfg.l : cfg.n + (s + 1) * cfg.l;
    }
    long ms() const { return (long)R_mem * cfg.m; }
    // device row tables: for s in 1..H, [act rows (R_act_max) | obs rows (p)];
    // row H+1 holds the identity rows and the caller's obs rows of oic_enks_update
    int* act_rows(int s) const { return at<int>(lay.rowtab) + (size_t)s * (R_act_max + p); }
    int* obs_rows(int s) const { return act_rows(s) + R_act_max; }
};

namespace {

// The plan's values, rules resolved.
int cnn_ctas(const oic_handle* h) { return h->plan.cnn_ctas > 0 ? h->plan.cnn_ctas : h->n_sm; }
int update_ctas(const oic_handle* h) { return h->plan.update_ctas > 0 ? h->plan.update_ctas : 148; }
int plan_splits(const oic_handle* h, int rule)
{
    const int s = h->plan.stats_splits > 0 ? h->plan.stats_splits : rule;
    return s < h->splits_max ? s : h->splits_max;
}

// Runs one kernel launch of stage `stage`, counting it and, when the stage is
// being profiled, bracketing it with CUDA events on the bound stream (while a
// step graph is being captured: with capture-time events that become the
// graph's record nodes).
template <typename F>
void run_stage(oic_handle* h, int stage, F&& launch)
{
    const int seen = h->stage_seen[stage]++;
    if (h->capturing != nullptr) {
        StepGraph& G = *h->capturing;
        cudaEvent_t e[2] = {nullptr, nullptr};
        const bool rec = ((G.mask >> stage) & 1u) && seen % G.every == G.phase &&
                         cudaEventCreate(&e[0]) == cudaSuccess && cudaEventCreate(&e[1]) == cudaSuccess;
        if (rec) cudaEventRecord(e[0], h->st);
        launch();
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if (rec) {
            cudaEventRecord(e[1], h->st);
            G.cap_ev.push_back(e[0]);
            G.cap_ev.push_back(e[1]);
            G.stage.push_back(stage);
        } else {
            if (e[0]) cudaEventDestroy(e[0]);
            if (e[1]) cudaEventDestroy(e[1]);
        }
        return;
    }
    Profiler& P = h->prof;
    const bool rec = P.on && ((P.mask >> stage) & 1u) && seen % P.every == P.phase && P.used < P.max;
    if (rec) cudaEventRecord(P.ev[2 * P.used], h->st);
    launch();
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (rec) {
        cudaEventRecord(P.ev[2 * P.used + 1], h->st);
        P.stage[P.used] = stage;
        ++P.used;
    }
}

bool valid_config(const oic_config* c)
{
    if (!c) return false;
    if (c->n < 1 || c->m < 4 || c->m % 4 != 0 || c->l < 1 || c->N < 2 || c->H < 1) return false;
    if (c->n_layers < 1 || c->n_layers > OIC_MAX_LAYERS) return false;
    if (c->channels[0] != 2 || c->channels[c->n_layers] != 1) return false;
    for (int k = 0; k <= c->n_layers; ++k)
        if (c->channels[k] < 1 || c->channels[k] > 256) return false;
    if (c->precision != OIC_PREC_FP32 && c->precision != OIC_PREC_MIXED) return false;
    if (c->noise_mode != OIC_NOISE_HOST && c->noise_mode != OIC_NOISE_PHILOX) return false;
    const long p = (long)c->n + c->l;
    if (p > 144) return false;                  // the sizes the gain and covariance kernels are built and tested for
    if ((long)c->n * c->m > (1L << 26) || (long)c->N * c->m > (1L << 28)) return false;
    if (c->m > 128) return false;                // analysis tiles hold one member row of <= 128 columns
    return true;
}

size_t noise_count(const oic_config* c, int nc = 0)
{
    const size_t N = c->N, n = c->n, m = c->m, l = c->l, H = c->H;
    return N * l * m + H * N * (l * m + n * m + l * m + (size_t)nc * m);
}

void compute_layout(oic_handle* h)
{
    const oic_config& c = h->cfg;
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        const size_t off = cur;
        cur += align_up(bytes > 0 ? bytes : 1, 256);
        return off;
    };
    const size_t n = c.n, m = c.m, l = c.l, N = c.N, H = c.H, p = h->p;
    const size_t Ra = h->R_act_max;
    Layout& L = h->lay;
    L.w = take(sizeof(float) * h->w.size());
    L.b = take(sizeof(float) * h->b.size());
    L.B = take(sizeof(float) * n * l);
    {
        size_t tc_bytes = 0;
        h->wtc_off.assign(h->L, SIZE_MAX);
        for (int k = 1; k + 1 < h->L; ++k)
            if (conv_tc_supported(c.channels[k], c.channels[k + 1], c.m)) {
                h->wtc_off[k] = tc_bytes;
                tc_bytes += align_up(conv_tc_packed_bytes(c.channels[k]), 256);
            }
        L.wtc = take(tc_bytes);
        L.wfused = take(h->fused ? cnn_fused_packed_bytes() : 0);
    }
    {
        // mixed-precision CNN: per layer packed BF16 tiles and biases padded to CO
        size_t wb = 0, bb = 0;
        h->w16_off.assign(h->L, 0);
        h->b16_off.assign(h->L, 0);
        if (h->bf16) {
            const int C = c.channels[1];
            for (int k = 0; k < h->L; ++k) {
                const int CI = k == 0 ? 16 : C, CO = k + 1 == h->L ? 16 : C;
                h->w16_off[k] = wb;
                wb += align_up(bf16_layer_bytes(CI, CO), 256);
                h->b16_off[k] = bb;
                bb += align_up(sizeof(float) * CO, 256);
            }
        }
        L.w16 = take(wb);
        L.b16 = take(bb);
        L.act16_in = take(h->bf16 ? bf16_act_bytes(c.N, c.n, c.m, 16) : 0);
    }
    L.E = take(sizeof(float) * N * h->R_mem * m);
    // per-layer activations: FP32 [N][C][n][m], or BF16 operand rows in the
    // mixed-precision mode (smaller)
    const size_t act_bytes = h->bf16 ? bf16_act_bytes(c.N, c.n, c.m, c.channels[1]) : sizeof(float) * N * h->Cmax * n * m;
    L.act0 = take(act_bytes);
    L.act1 = take(act_bytes);
    L.part1 = take(sizeof(float) * (size_t)h->splits_max * (Ra + p) * m);
    L.part2 = take(sizeof(float) * (size_t)h->splits_max * (Ra + p) * p);
    L.S1 = take(sizeof(double) * (Ra + p) * m);           // FP64 in the mixed mode
    L.S1T = take(sizeof(double) * p * m);                 // the observed rows' sums, transposed
    L.D = take(sizeof(float) * N * p * m);
    L.C = take(sizeof(double) * (Ra + p) * p);
    L.K = take(sizeof(float) * Ra * p);
    L.cyy32 = take(c.precision == OIC_PREC_MIXED ? 0 : gain_cyy32_bytes((int)p));
    L.L64 = take(c.precision == OIC_PREC_MIXED ? sizeof(double) * (p * p + p) : 0);
    // tensor-core anomaly products: the pre-split observation tiles
    L.tB = take(stats_tc_supported(c.m, (int)p) ? stats_tc_bbytes(c.N, (int)p, c.m) : 0);
    // tensor-core update: gain tiles and the transposed innovations
    const bool utc = stats_tc_supported(c.m, (int)p) && update_tc_supported(c.m, (int)p);
    L.tAop = take(utc ? update_tc_abytes((int)Ra, (int)p) : 0);
    L.tBd = take(utc ? update_tc_bbytes(c.N, c.m, (int)p) : 0);
    L.ctr = take(sizeof(unsigned long long));            // Philox solve index
    L.rowtab = take(sizeof(int) * (H + 2) * (Ra + p));
    L.status = take(64);
    L.selftest = take(64);
    L.cG = take(sizeof(float) * h->cG.size());
    L.ccols = take(sizeof(int) * h->ccols.size());
    L.ch = take(sizeof(float) * h->ch.size());
    L.plantX = take(sizeof(float) * n * m);
    L.plantU = take(sizeof(float) * l * m);
    L.plantTmp = take(sizeof(float) * n * m);
    L.xk = take(sizeof(float) * n * m);
    L.uprev = take(sizeof(float) * l * m);
    L.xref = take(sizeof(float) * (H + 1) * n * m);
    L.uref = take(sizeof(float) * l * m);
    L.noise = take(sizeof(float) * h->noise_n);
    L.uhat = take(sizeof(float) * (H + 1) * l * m);
    L.xhat = take(sizeof(float) * (H + 1) * n * m);
    L.uapp = take(sizeof(float) * l * m);
    L.xnext = take(sizeof(float) * n * m);
    L.total = cur;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

oic_status last_cuda()
{
    return cudaGetLastError() == cudaSuccess ? OIC_OK : OIC_ECUDA;
}

// X_next[b] = CNN_theta(X[b], U[b]) for b < Nb, member strides x_ms / u_ms / o_ms.
// ua: the control advance U_t = U_{t-1} + W, done by the fused FP32 CNN kernel
// while it reads U (cnn_advances_u); the caller launches it otherwise.  The
// BF16 path keeps the separate launch: the advance inside its first kernel
// measured slower at 128 x 128 (13.17 against 13.39 control steps/s on one box).
bool cnn_advances_u(const oic_handle* h) { return h->fused; }

void cnn_forward(oic_handle* h, int Nb, const float* X, long x_ms, const float* U, long u_ms,
                 float* Xout, long o_ms, UAdvance ua = UAdvance())
{
    const oic_config& c = h->cfg;
    if (h->bf16) {
        Bf16Net net;
        net.n_layers = h->L;
        net.C = c.channels[1];
        for (int k = 0; k < h->L; ++k) {
            net.w[k] = h->at<char>(h->lay.w16) + h->w16_off[k];
            net.b[k] = reinterpret_cast<const float*>(h->at<char>(h->lay.b16) + h->b16_off[k]);
        }
        net.act_in = h->at<char>(h->lay.act16_in);
        net.act[0] = h->at<char>(h->lay.act0);
        net.act[1] = h->at<char>(h->lay.act1);
        run_stage(h, OIC_STAGE_CNN_BF16, [&] {
            launch_bf16_forward(net, X, x_ms, U, u_ms, Xout, o_ms, h->at<float>(h->lay.B), Nb, c.n, c.m, c.l,
                                c.residual_scale, cnn_ctas(h), h->at<int>(h->lay.status), h->st);
        });
        return;
    }
    if (h->fused) {
        const float* b = h->at<float>(h->lay.b);
        const int C = c.channels[1];
        run_stage(h, OIC_STAGE_CNN_FUSED, [&] {
            launch_cnn_fused(X, x_ms, U, u_ms, Xout, o_ms, h->at<float>(h->lay.B), Nb, c.n, c.m, c.l, b,
                             b + C, b + 2 * C, h->at<char>(h->lay.wfused), c.residual_scale, cnn_ctas(h),
                             h->at<int>(h->lay.status), h->st, ua);
        });
        return;
    }
    float* a = h->at<float>(h->lay.act0);
    float* z = h->at<float>(h->lay.act1);
    run_stage(h, OIC_STAGE_CNN_INPUT, [&] {
        launch_cnn_input(X, x_ms, U, u_ms, h->at<float>(h->lay.B), a, Nb, c.n, c.m, c.l, h->st);
    });
    const float* w = h->at<float>(h->lay.w);
    const float* b = h->at<float>(h->lay.b);
    for (int k = 0; k < h->L - 1; ++k) {
        const int cin = c.channels[k], cout = c.channels[k + 1];
        const size_t toff = h->wtc_off[k];
        run_stage(h, k == 0 ? OIC_STAGE_CONV_FIRST : OIC_STAGE_CONV_HIDDEN, [&] {
            if (toff != SIZE_MAX)
                launch_conv_tc(a, z, h->at<char>(h->lay.wtc) + toff, b, cout, Nb, c.n, c.m, cnn_ctas(h),
                               h->at<int>(h->lay.status), h->st);
            else
                launch_conv_hidden(a, cin, z, cout, Nb, c.n, c.m, w, b, h->st);
        });
        w += (size_t)cin * cout * 9;
        b += cout;
        float* t = a; a = z; z = t;
    }
    run_stage(h, OIC_STAGE_CONV_OUT, [&] {
        launch_conv_out_residual(a, c.channels[h->L - 1], X, x_ms, Xout, o_ms, Nb, c.n, c.m, w, b,
                                 c.residual_scale, h->st);
    });
}

// One ensemble Kalman analysis on rows `act` / `obs` of the ensemble E.
void analysis(oic_handle* h, float* E, long ms, RowSet act, RowSet obs, ObsNoise V, const float* Yx,
              const float* Yu, int n_yx)
{
    const oic_config& c = h->cfg;
    float* part1 = h->at<float>(h->lay.part1);
    float* part2 = h->at<float>(h->lay.part2);
    float* S1 = h->at<float>(h->lay.S1);
    float* S1T = h->at<float>(h->lay.S1T);
    float* D = h->at<float>(h->lay.D);
    double* C = h->at<double>(h->lay.C);
    float* Kt = h->at<float>(h->lay.K);
    const int R = act.count, p = obs.count, M = R + p;
    const bool mixed = c.precision == OIC_PREC_MIXED;
    const bool tcs = stats_tc_supported(c.m, p);
    const bool utc = tcs && update_tc_supported(c.m, p);
    float* Bd = utc ? h->at<float>(h->lay.tBd) : nullptr;
    // the FP32 gain stages Sigma^Y from an FP32 copy in its own layout
    float* cyy32 = !mixed && gain_cyy32_bytes(p) <= gain_cyy32_bytes(h->p) ? h->at<float>(h->lay.cyy32) : nullptr;
    if (tcs) {
        const int splits = plan_splits(h, stats_tc_splits(M, c.N));
        run_stage(h, OIC_STAGE_COV, [&] {
            launch_stats_tc(E, ms, c.N, c.m, act, obs, V, Yx, Yu, n_yx, h->at<float>(h->lay.tB), part1, part2,
                            utc ? nullptr : D, Bd, splits, h->at<int>(h->lay.status), h->st);
        });
        run_stage(h, OIC_STAGE_MEANS, [&] { launch_s1_reduce(part1, splits, M, c.m, S1, h->st, S1T, R, mixed); });
        run_stage(h, OIC_STAGE_COV_REDUCE, [&] {
            launch_cov_finalize(part2, S1, splits, R, p, c.m, c.N, C, h->st, mixed, 1.0, S1T, cyy32);
        });
    } else {
        const int splits = plan_splits(h, stats_splits(R, p, c.N));
        run_stage(h, OIC_STAGE_COV, [&] {
            launch_stats(E, ms, c.N, c.m, act, obs, V, Yx, Yu, n_yx, part1, part2, D, splits, h->st);
        });
        run_stage(h, OIC_STAGE_MEANS, [&] { launch_s1_reduce(part1, splits, M, c.m, S1, h->st, S1T, R, mixed); });
        run_stage(h, OIC_STAGE_COV_REDUCE, [&] {
            launch_cov_finalize(part2, S1, splits, R, p, c.m, c.N, C, h->st, mixed, 1.0, S1T, cyy32);
        });
    }
    run_stage(h, OIC_STAGE_GAIN, [&] {
        if (mixed)
            launch_gain64(C, R, p, h->at<double>(h->lay.L64), h->at<int>(h->lay.status) + 1, Kt,
                          h->at<int>(h->lay.status), h->st);
        else
            launch_gain(C, R, p, Kt, h->at<int>(h->lay.status), h->st,
                        utc ? h->at<float>(h->lay.tAop) : nullptr, cyy32);
    });
    if (utc)
        run_stage(h, OIC_STAGE_UPDATE, [&] {
            launch_update_tc(E, ms, c.N, c.m, act, Kt, p, h->at<float>(h->lay.tAop), update_ctas(h), Bd,
                             h->at<int>(h->lay.status),
                             h->st, mixed);                // the FP32 gain writes the tiles itself
        });
    else
        run_stage(h, OIC_STAGE_UPDATE, [&] { launch_update(E, ms, c.N, c.m, act, Kt, p, D, h->st); });
}

// Algorithm 1's optional covariance steps (the predicted and the updated state
// covariance): where to write
// them and the scratch the products use.
struct CovOut {
    double lambda = 1.0;
    double* pred = nullptr;          // [H][R_max][R_max] slots, compact R_of(s)^2 each
    double* post = nullptr;
    char* scratch = nullptr;
};

// part1 / part2 / S1 of the row covariance of R kept rows (no state rows,
// the kept rows as the observed side of the anomaly products)
struct CovScratch {
    size_t part1, part2, S1, total;
};
CovScratch cov_scratch(const oic_handle* h)
{
    CovScratch c{0, 0, 0, 0};
    size_t p1 = 0, p2 = 0, s1 = 0;
    for (int s = 1; s <= h->cfg.H; ++s) {
        const size_t R = h->R_of(s), sp = stats_splits(0, (int)R, h->cfg.N);
        p1 = std::max(p1, sp * R * h->cfg.m);
        p2 = std::max(p2, sp * R * R);
        s1 = std::max(s1, R * h->cfg.m);
    }
    c.part1 = 0;
    c.part2 = align_up(sizeof(float) * p1, 256);
    c.S1 = c.part2 + align_up(sizeof(float) * p2, 256);
    c.total = c.S1 + align_up(sizeof(double) * s1, 256);
    return c;
}

// out = (lambda / N) sum_i (E^i[rows] - mean)(E^i[rows] - mean)^T over the
// kept rows `rows` (pooled over the m columns), FP64 split sums and mean
// correction.
void ensemble_cov(oic_handle* h, const float* E, long ms, RowSet rows, const CovOut& co, double* out)
{
    const oic_config& c = h->cfg;
    const CovScratch cs = cov_scratch(h);
    float* part1 = reinterpret_cast<float*>(co.scratch + cs.part1);
    float* part2 = reinterpret_cast<float*>(co.scratch + cs.part2);
    double* S1 = reinterpret_cast<double*>(co.scratch + cs.S1);
    const int R = rows.count;
    const int splits = stats_splits(0, R, c.N);
    RowSet none{rows.rows, 0};
    run_stage(h, OIC_STAGE_COV_OUT, [&] {
        launch_stats(E, ms, c.N, c.m, none, rows, ObsNoise(), nullptr, nullptr, 0, part1, part2,
                     nullptr, splits, h->st);
    });
    run_stage(h, OIC_STAGE_COV_OUT, [&] { launch_s1_reduce(part1, splits, R, c.m, S1, h->st, nullptr, 0, true); });
    run_stage(h, OIC_STAGE_COV_OUT, [&] {
        launch_cov_finalize(part2, S1, splits, 0, R, c.m, c.N, out, h->st, true, co.lambda / c.N);
    });
}

oic_status solve_impl(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                      const float* U_ref, const float* noise, float* U_hat, float* X_hat, const CovOut* cov = nullptr,
                      float* u0a = nullptr, float* u0b = nullptr)
{
    const oic_config& c = h->cfg;
    const size_t N = c.N, n = c.n, m = c.m, l = c.l, H = c.H;
    for (int& v : h->stage_seen) v = 0;
    // The solve's random numbers, segments W0 | W | V_X | V_U | eps of the
    // noise layout.  Device mode: each consumer draws its elements in place
    // from the Philox stream (the numbers the noise kernel would write, bit for
    // bit); with OIC_NOISE_BUFFER set the noise kernel writes the whole stream
    // to the buffer first and the consumers read it.  The solve index
    // advances after the solve's last draw.
    const size_t e0 = N * l * m, e1 = e0 + H * N * l * m, e2 = e1 + H * N * n * m,
                 e3 = e2 + H * N * l * m, e4 = e3 + H * N * (size_t)h->nc * m;
    const bool philox = c.noise_mode == OIC_NOISE_PHILOX;
    const bool in_place = philox && getenv("OIC_NOISE_BUFFER") == nullptr;
    unsigned long long* ctr = h->at<unsigned long long>(h->lay.ctr);
    if (philox && !in_place) {
        const size_t ends[5] = {e0, e1, e2, e3, e4};
        const float sig[5] = {(float)c.sigma_w, (float)c.sigma_w, (float)c.sigma_vx, (float)c.sigma_vu, h->c_sigma};
        float* buf = h->at<float>(h->lay.noise);
        run_stage(h, OIC_STAGE_NOISE, [&] {
            launch_philox_noise(buf, h->noise_n, c.seed, ctr, ends, sig, h->nc > 0 ? 5 : 4, h->st, false);
        });
        noise = buf;
    }
    auto segment = [&](size_t start, float sigma) {
        NoiseSrc s;
        if (in_place) {
            s.ctr = ctr;
            s.seed = c.seed;
            s.base = start;
            s.sigma = sigma;
        } else {
            s.buf = noise + start;
        }
        return s;
    };
    float* E = h->at<float>(h->lay.E);
    const long ms = h->ms();

    run_stage(h, OIC_STAGE_INIT, [&] {
        launch_ensemble_init(E, ms, c.N, c.n, c.m, c.l, h->xrow(0), h->urow(0), X_k, U_prev,
                             segment(0, (float)c.sigma_w), h->st);
    });
    for (int s = 1; s <= c.H; ++s) {
        // prediction, Eq. (prediction-samplewise): X̄_t = f_CNN(X̄_{t-1}) + W̄_{t-1}
        const NoiseSrc Ws = segment(e0 + (s - 1) * N * l * m, (float)c.sigma_w);
        UAdvance ua;
        if (cnn_advances_u(h)) {
            ua.next = E + (size_t)h->urow(s) * m;
            ua.w = Ws;
        }
        cnn_forward(h, c.N, E + (size_t)h->xrow(s - 1) * m, ms, E + (size_t)h->urow(s - 1) * m, ms,
                    E + (size_t)h->xrow(s) * m, ms, ua);
        if (!cnn_advances_u(h))
            run_stage(h, OIC_STAGE_U_ADVANCE, [&] {
                launch_u_advance(E, ms, c.N, c.m, c.l, h->urow(s - 1), h->urow(s), Ws, h->st);
            });
        // constraint rows z_t = phi(g(X_t, U_t)) + eps_t (reference 0)
        if (h->nc > 0)
            run_stage(h, OIC_STAGE_CONSTRAINT, [&] {
                launch_constraint_obs(E, ms, c.N, c.m, c.n, h->xrow(s), h->urow(s), h->zrow, h->nc,
                                      h->at<float>(h->lay.cG), h->at<int>(h->lay.ccols), h->nk,
                                      h->at<float>(h->lay.ch), h->c_alpha, h->c_beta,
                                      segment(e3 + (s - 1) * N * (size_t)h->nc * m, h->c_sigma), h->st);
            });
        // analysis at t = k + s with Ybar_t = [X_ref[s]; U_ref; 0]
        RowSet act{h->act_rows(s), h->R_of(s)};
        RowSet obs{h->obs_rows(s), h->p, h->nc};
        ObsNoise V;
        V.a = segment(e1 + (s - 1) * N * n * m, (float)c.sigma_vx);
        V.b = segment(e2 + (s - 1) * N * l * m, (float)c.sigma_vu);
        V.pa = c.n;
        const size_t slot = (size_t)(s - 1) * h->R_act_max * h->R_act_max;
        if (cov && cov->pred) ensemble_cov(h, E, ms, act, *cov, cov->pred + slot);     // Sigma^X_{t|t-1}
        analysis(h, E, ms, act, obs, V, X_ref + (size_t)s * n * m, U_ref, c.n);
        if (cov && cov->post) ensemble_cov(h, E, ms, act, *cov, cov->post + slot);     // Sigma^X_{t|t}
    }
    // the smoothed means (Û_k also to u0a / u0b where given); the first launch
    // also advances the solve index, every draw of the solve being done
    run_stage(h, OIC_STAGE_BLOCK_MEANS, [&] {
        launch_block_means(E, ms, c.N, c.m, h->urow(0), c.l, c.H + 1, U_hat, h->st, philox ? ctr : nullptr, u0a,
                           u0b);
    });
    if (X_hat)
        run_stage(h, OIC_STAGE_BLOCK_MEANS, [&] {
            launch_block_means(E, ms, c.N, c.m, 0, c.n, c.H + 1, X_hat, h->st);
        });
    return last_cuda();
}

oic_status step_impl(oic_handle* h, const float* X_ref, const float* U_ref, const float* noise,
                     float* U_applied, float* X_next)
{
    const oic_config& c = h->cfg;
    const size_t n = c.n, m = c.m;
    float* uhat = h->at<float>(h->lay.uhat);
    float* pX = h->at<float>(h->lay.plantX);
    float* pU = h->at<float>(h->lay.plantU);
    float* tmp = h->at<float>(h->lay.plantTmp);
    // the solve's block means also write Û_k to the plant's control and to
    // U_applied (the solve read U_prev = pU at its start)
    oic_status s = solve_impl(h, pX, pU, X_ref, U_ref, noise, uhat,
                              h->full() ? h->at<float>(h->lay.xhat) : nullptr, nullptr, pU, U_applied);
    if (s != OIC_OK) return s;
    // Algorithm 1, end of the control step: apply U_k = Û_{k|k:k+H} to the plant, then
    // X_k <- X_{k+1} (and X_next) in one launch
    cnn_forward(h, 1, pX, 0, uhat, 0, tmp, 0);
    launch_copy2(tmp, pX, X_next, (int)(n * m), h->st);
    return last_cuda();
}

// Captures step_impl on the workspace buffers into G (event nodes for the
// stages in mask).  A failed capture leaves G.failed set and the caller runs
// the step eagerly.
bool capture_step(oic_handle* h, StepGraph& G, unsigned mask)
{
    G.reset();
    G.mask = mask;
    G.every = h->prof.every;
    G.phase = h->prof.phase;
    const Layout& L = h->lay;
    const unsigned long long l0 = g_launches.load();
    h->capturing = &G;
    oic_status s = OIC_ECUDA;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        s = step_impl(h, h->at<float>(L.xref), h->at<float>(L.uref), h->at<float>(L.noise), h->at<float>(L.uapp),
                      h->at<float>(L.xnext));
        if (cudaStreamEndCapture(h->st, &G.g) != cudaSuccess) s = OIC_ECUDA;
    }
    h->capturing = nullptr;
    G.launches = g_launches.load() - l0;
    g_launches.fetch_sub(G.launches);                     // captured, not run
    if (s != OIC_OK || G.g == nullptr ||
        cudaGraphInstantiate(&G.x, G.g, 0) != cudaSuccess) {
        cudaGetLastError();
        G.reset();
        G.failed = true;
        return false;
    }
    if (!G.cap_ev.empty()) {
        size_t n = 0;
        cudaGraphGetNodes(G.g, nullptr, &n);
        std::vector<cudaGraphNode_t> all(n);
        cudaGraphGetNodes(G.g, all.data(), &n);
        G.node.assign(G.cap_ev.size(), nullptr);
        for (cudaGraphNode_t nd : all) {
            cudaGraphNodeType t;
            cudaEvent_t e = nullptr;
            if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
            if (cudaGraphEventRecordNodeGetEvent(nd, &e) != cudaSuccess) continue;
            for (size_t k = 0; k < G.cap_ev.size(); ++k)
                if (G.cap_ev[k] == e) G.node[k] = nd;
        }
        for (cudaGraphNode_t nd : G.node)
            if (nd == nullptr) {
                G.reset();
                G.failed = true;
                return false;
            }
    }
    return true;
}

// One control step through the step graph; false when no graph can be used
// (the caller then runs step_impl eagerly).
bool run_step_graph(oic_handle* h)
{
    if (h->cfg.noise_mode != OIC_NOISE_PHILOX || getenv("OIC_NO_GRAPH") != nullptr) return false;
    Profiler& P = h->prof;
    const bool prof = P.on && P.mask != 0;
    StepGraph* G = &h->sg[prof ? 1 : 0];
    if (prof && G->x && (G->mask != P.mask || G->every != P.every || G->phase != P.phase)) G->reset();
    if (!G->x && !G->failed) capture_step(h, *G, prof ? P.mask : 0);
    if (!G->x) return false;
    if (prof) {
        const int pairs = (int)G->stage.size();
        if (P.used + pairs > P.max) return false;         // out of profiler slots: eager, untimed
        for (int k = 0; k < pairs; ++k) {
            if (cudaGraphExecEventRecordNodeSetEvent(G->x, G->node[2 * k], P.ev[2 * (P.used + k)]) != cudaSuccess ||
                cudaGraphExecEventRecordNodeSetEvent(G->x, G->node[2 * k + 1], P.ev[2 * (P.used + k) + 1]) !=
                    cudaSuccess)
                return false;
            P.stage[P.used + k] = G->stage[k];
        }
        P.used += pairs;
    }
    if (cudaGraphLaunch(G->x, h->st) != cudaSuccess) return false;
    g_launches.fetch_add(G->launches, std::memory_order_relaxed);
    return true;
}

// ---------------------------------------------------------------- plans
// Plans chosen by oic_autotune, by problem shape (process-wide).
std::mutex g_plan_mu;
std::map<std::string, oic_plan> g_plan_cache;

std::string plan_key(const oic_handle* h)
{
    const oic_config& c = h->cfg;
    std::string k = std::to_string(c.n) + "x" + std::to_string(c.m) + "/l" + std::to_string(c.l) + "/N" +
                    std::to_string(c.N) + "/H" + std::to_string(c.H) + "/c";
    for (int i = 0; i <= c.n_layers; ++i) k += std::to_string(c.channels[i]) + ",";
    k += "/pr" + std::to_string(c.precision) + "/fh" + std::to_string(c.keep_full_history) + "/nm" +
         std::to_string(c.noise_mode) + "/nc" + std::to_string(h->nc) + "/sm" + std::to_string(h->n_sm);
    return k;
}

// The covariance products' rule at the last assimilation time (the largest
// row count).
int rule_splits(const oic_handle* h)
{
    const int R = h->R_of(h->cfg.H), p = h->p;
    return stats_tc_supported(h->cfg.m, p) ? stats_tc_splits(R + p, h->cfg.N) : stats_splits(R, p, h->cfg.N);
}

oic_plan effective_plan(const oic_handle* h)
{
    oic_plan e;
    e.stats_splits = plan_splits(h, rule_splits(h));
    e.update_ctas = update_ctas(h);
    e.cnn_ctas = cnn_ctas(h);
    return e;
}

oic_plan plan_limits(const oic_handle* h)
{
    oic_plan l;
    l.stats_splits = h->splits_max;
    l.update_ctas = 148;
    l.cnn_ctas = h->n_sm;
    return l;
}

void drop_step_graphs(oic_handle* h)
{
    h->sg[0].reset();
    h->sg[1].reset();
}

oic_status read_status(oic_handle* h)
{
    int dev = 0;
    OIC_CUDA_OK(cudaMemcpyAsync(&dev, h->at<int>(h->lay.status), sizeof(int), cudaMemcpyDeviceToHost,
                                h->st));
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    if (dev != DEV_OK) {
        OIC_CUDA_OK(cudaMemsetAsync(h->at<int>(h->lay.status), 0, sizeof(int), h->st));
        OIC_CUDA_OK(cudaStreamSynchronize(h->st));
        return dev == DEV_NOTSPD ? OIC_ENOTSPD : OIC_ETIMEOUT;
    }
    return OIC_OK;
}

}  // namespace

extern "C" {

size_t oic_noise_floats(const oic_config* cfg) { return valid_config(cfg) ? noise_count(cfg) : 0; }

size_t oic_handle_noise_floats(const oic_handle* h) { return h ? h->noise_n : 0; }

oic_status oic_create(const oic_config* cfg, const float* conv_w, const float* conv_b, const float* B,
                      oic_handle** out)
{
    return oic_create_constrained(cfg, conv_w, conv_b, B, nullptr, out);
}

oic_status oic_create_constrained(const oic_config* cfg, const float* conv_w, const float* conv_b,
                                  const float* B, const oic_constraints* cons, oic_handle** out)
{
    if (!out) return OIC_EINVAL;
    *out = nullptr;
    if (!valid_config(cfg) || !conv_w || !conv_b || !B) return OIC_EINVAL;
    const int nc = cons ? cons->c : 0;
    if (nc < 0 || (long)cfg->n + cfg->l + nc > 144) return OIC_EINVAL;
    if (nc > 0 && (!cons->Gx || !cons->Gu || !cons->h || !(cons->alpha > 0.0) || !(cons->beta > 0.0) ||
                   !(cons->sigma_z >= 0.0)))
        return OIC_EINVAL;
    oic_handle* h = new (std::nothrow) oic_handle();
    if (!h) return OIC_ENOMEM;
    h->cfg = *cfg;
    const oic_config& c = h->cfg;
    h->L = c.n_layers;
    size_t nw = 0, nb = 0;
    for (int k = 0; k < h->L; ++k) {
        nw += (size_t)c.channels[k] * c.channels[k + 1] * 9;
        nb += c.channels[k + 1];
        if (k > 0 && c.channels[k] > h->Cmax) h->Cmax = c.channels[k];
    }
    try {
        h->w.assign(conv_w, conv_w + nw);
        h->b.assign(conv_b, conv_b + nb);
        h->B.assign(B, B + (size_t)c.n * c.l);
    } catch (...) {
        delete h;
        return OIC_ENOMEM;
    }
    h->q = c.n + 2 * c.l;
    h->nc = nc;
    h->p = c.n + c.l + nc;
    h->R_mem = h->full() ? (c.H + 1) * (c.n + c.l) : 2 * c.n + (c.H + 1) * c.l;
    h->zrow = h->R_mem;                       // constraint block after the state rows
    h->R_mem += nc;
    if (nc > 0) {
        // keep the columns of [Gx Gu] that are not all zero, in order
        const int nl = c.n + c.l;
        for (int a = 0; a < nl; ++a) {
            bool any = false;
            for (int r = 0; r < nc; ++r)
                any = any || (a < c.n ? cons->Gx[(size_t)r * c.n + a] : cons->Gu[(size_t)r * c.l + (a - c.n)]) != 0.f;
            if (any) h->ccols.push_back(a);
        }
        h->nk = (int)h->ccols.size();
        h->cG.assign((size_t)nc * (h->nk > 0 ? h->nk : 1), 0.f);
        for (int r = 0; r < nc; ++r)
            for (int k = 0; k < h->nk; ++k) {
                const int a = h->ccols[k];
                h->cG[(size_t)r * h->nk + k] =
                    a < c.n ? cons->Gx[(size_t)r * c.n + a] : cons->Gu[(size_t)r * c.l + (a - c.n)];
            }
        h->ch.assign(cons->h, cons->h + nc);
        h->c_alpha = (float)cons->alpha;
        h->c_beta = (float)cons->beta;
        h->c_sigma = (float)cons->sigma_z;
    }
    h->Ubase = h->full() ? (c.H + 1) * c.n : 2 * c.n;
    h->R_act_max = h->R_of(c.H);
    h->splits_max = stats_splits(1, h->p, c.N);
    if (stats_tc_splits(1, c.N) > h->splits_max) h->splits_max = stats_tc_splits(1, c.N);
    h->noise_n = noise_count(&c, nc);
    h->bf16 = c.precision == OIC_PREC_MIXED && bf16_supported(c.n_layers, c.channels, c.m);
    h->fused = !h->bf16 && cnn_fused_supported(c.n_layers, c.channels, c.n, c.m, c.l) &&
               getenv("OIC_NO_FUSED_CNN") == nullptr;
    compute_layout(h);
    *out = h;
    return OIC_OK;
}

size_t oic_workspace_bytes(const oic_handle* h) { return h ? h->lay.total : 0; }

int oic_max_rows(const oic_handle* h) { return h ? h->R_act_max : 0; }

oic_status oic_bind(oic_handle* h, void* dev_workspace, size_t bytes, void* cuda_stream)
{
    if (!h || !dev_workspace) return OIC_EINVAL;
    if (bytes < h->lay.total) return OIC_ENOMEM;
    if (reinterpret_cast<uintptr_t>(dev_workspace) % 256 != 0) return OIC_EINVAL;
    h->ws = static_cast<char*>(dev_workspace);
    h->ws_bytes = bytes;
    h->st = static_cast<cudaStream_t>(cuda_stream);
    const oic_config& c = h->cfg;
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.w), h->w.data(), sizeof(float) * h->w.size(),
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.b), h->b.data(), sizeof(float) * h->b.size(),
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.B), h->B.data(), sizeof(float) * h->B.size(),
                                cudaMemcpyHostToDevice, h->st));
    {
        int dev = 0;
        OIC_CUDA_OK(cudaGetDevice(&dev));
        OIC_CUDA_OK(cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev));
        if (conv_tc_configure() != 0) return OIC_ECUDA;
        const float* wl = h->w.data();
        for (int k = 0; k < h->L; ++k) {
            const int cin = c.channels[k], cout = c.channels[k + 1];
            if (h->wtc_off[k] != SIZE_MAX) {
                std::vector<unsigned char> pk(conv_tc_packed_bytes(cout));
                conv_tc_pack_weights(wl, cout, pk.data());
                OIC_CUDA_OK(cudaMemcpy(h->at<char>(h->lay.wtc) + h->wtc_off[k], pk.data(), pk.size(),
                                       cudaMemcpyHostToDevice));
            }
            wl += (size_t)cin * cout * 9;
        }
        if (h->fused) {
            const int C = c.channels[1];
            const float* w1 = h->w.data();
            const float* w2 = w1 + (size_t)2 * C * 9;
            const float* w3 = w2 + (size_t)C * C * 9;
            std::vector<unsigned char> pk(cnn_fused_packed_bytes());
            cnn_fused_pack_weights(w1, w2, w3, pk.data());
            OIC_CUDA_OK(cudaMemcpy(h->at<char>(h->lay.wfused), pk.data(), pk.size(), cudaMemcpyHostToDevice));
        }
        if (h->bf16) {
            const int C = c.channels[1];
            const float* wl2 = h->w.data();
            const float* bl = h->b.data();
            for (int k = 0; k < h->L; ++k) {
                const int cin = c.channels[k], cout = c.channels[k + 1];
                const int CI = k == 0 ? 16 : C, CO = k + 1 == h->L ? 16 : C;
                std::vector<unsigned char> pk(bf16_layer_bytes(CI, CO));
                bf16_pack_layer(wl2, cin, cout, CI, CO, pk.data());
                OIC_CUDA_OK(cudaMemcpy(h->at<char>(h->lay.w16) + h->w16_off[k], pk.data(), pk.size(),
                                       cudaMemcpyHostToDevice));
                std::vector<float> bp(CO, 0.f);
                for (int o = 0; o < cout; ++o) bp[o] = bl[o];
                OIC_CUDA_OK(cudaMemcpy(h->at<char>(h->lay.b16) + h->b16_off[k], bp.data(), sizeof(float) * CO,
                                       cudaMemcpyHostToDevice));
                wl2 += (size_t)cin * cout * 9;
                bl += cout;
            }
            // operand rows: the pad positions (and the first layer's zero
            // channels) are never written, so they must start at zero
            OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.act16_in), 0,
                                        bf16_act_bytes(c.N, c.n, c.m, 16), h->st));
            OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.act0), 0, bf16_act_bytes(c.N, c.n, c.m, C), h->st));
            OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.act1), 0, bf16_act_bytes(c.N, c.n, c.m, C), h->st));
        }
    }
    // row tables
    const int stride = h->R_act_max + h->p;
    std::vector<int> tab((size_t)(c.H + 2) * stride, 0);
    for (int s = 1; s <= c.H; ++s) {
        int* a = tab.data() + (size_t)s * stride;
        int* o = a + h->R_act_max;
        int r = 0;
        if (h->full()) {
            for (int t = 1; t <= s; ++t)
                for (int y = 0; y < c.n; ++y) a[r++] = t * c.n + y;
        } else {
            for (int y = 0; y < c.n; ++y) a[r++] = h->xrow(s) + y;
        }
        for (int t = 0; t <= s; ++t)
            for (int y = 0; y < c.l; ++y) a[r++] = h->urow(t) + y;
        for (int y = 0; y < c.n; ++y) o[y] = h->xrow(s) + y;
        for (int y = 0; y < c.l; ++y) o[c.n + y] = h->urow(s) + y;
        for (int y = 0; y < h->nc; ++y) o[c.n + c.l + y] = h->zrow + y;
    }
    int* gen = tab.data() + (size_t)(c.H + 1) * stride;
    for (int r = 0; r < h->R_act_max; ++r) gen[r] = r;
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<int>(h->lay.rowtab), tab.data(), sizeof(int) * tab.size(),
                                cudaMemcpyHostToDevice, h->st));
    if (h->nc > 0) {
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.cG), h->cG.data(), sizeof(float) * h->cG.size(),
                                    cudaMemcpyHostToDevice, h->st));
        if (h->nk > 0)
            OIC_CUDA_OK(cudaMemcpyAsync(h->at<int>(h->lay.ccols), h->ccols.data(), sizeof(int) * h->ccols.size(),
                                        cudaMemcpyHostToDevice, h->st));
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.ch), h->ch.data(), sizeof(float) * h->ch.size(),
                                    cudaMemcpyHostToDevice, h->st));
    }
    OIC_CUDA_OK(cudaMemsetAsync(h->at<int>(h->lay.status), 0, 64, h->st));
    OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.ctr), 0, sizeof(unsigned long long), h->st));
    h->sg[0].reset();
    h->sg[1].reset();
    if (!h->ev0) OIC_CUDA_OK(cudaEventCreate(&h->ev0));
    if (!h->ev1) OIC_CUDA_OK(cudaEventCreate(&h->ev1));
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    h->bound = true;
    h->plant_ready = false;
    return OIC_OK;
}

oic_status oic_reset(oic_handle* h, const float* X0, const float* U_prev)
{
    if (!h || !X0 || !U_prev) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const size_t n = h->cfg.n, m = h->cfg.m, l = h->cfg.l;
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantX), X0, sizeof(float) * n * m,
                                cudaMemcpyDeviceToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantU), U_prev, sizeof(float) * l * m,
                                cudaMemcpyDeviceToDevice, h->st));
    OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.ctr), 0, sizeof(unsigned long long), h->st));
    h->plant_ready = true;
    return OIC_OK;
}

oic_status oic_solve(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                     const float* U_ref, const float* noise, float* U_hat, float* X_hat)
{
    if (!h || !X_k || !U_prev || !X_ref || !U_ref || !U_hat) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    if (h->cfg.noise_mode == OIC_NOISE_HOST && (!noise || !aligned16(noise))) return OIC_EINVAL;
    if (X_hat && !h->full()) return OIC_EINVAL;
    OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
    oic_status s = solve_impl(h, X_k, U_prev, X_ref, U_ref, noise, U_hat, X_hat);
    OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
    return s;
}

size_t oic_cov_scratch_bytes(const oic_handle* h) { return h ? cov_scratch(h).total : 0; }

int oic_cov_rows(const oic_handle* h, int s)
{
    if (!h || s < 1 || s > h->cfg.H) return 0;
    return h->R_of(s);
}

oic_status oic_solve_cov(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                         const float* U_ref, const float* noise, float* U_hat, float* X_hat, double lambda,
                         double* Sigma_pred, double* Sigma_post, void* scratch, size_t scratch_bytes)
{
    if (!h || !X_k || !U_prev || !X_ref || !U_ref || !U_hat) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    if (h->cfg.noise_mode == OIC_NOISE_HOST && (!noise || !aligned16(noise))) return OIC_EINVAL;
    if (X_hat && !h->full()) return OIC_EINVAL;
    if ((Sigma_pred || Sigma_post) &&
        (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 255u) != 0 || scratch_bytes < cov_scratch(h).total))
        return OIC_EINVAL;
    CovOut co;
    co.lambda = lambda;
    co.pred = Sigma_pred;
    co.post = Sigma_post;
    co.scratch = static_cast<char*>(scratch);
    OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
    oic_status s = solve_impl(h, X_k, U_prev, X_ref, U_ref, noise, U_hat, X_hat, &co);
    OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
    return s;
}

oic_status oic_step(oic_handle* h, const float* X_ref, const float* U_ref, const float* noise,
                    float* U_applied, float* X_next)
{
    if (!h || !X_ref || !U_ref) return OIC_EINVAL;
    if (!h->bound || !h->plant_ready) return OIC_ESTATE;
    if (h->cfg.noise_mode == OIC_NOISE_HOST && (!noise || !aligned16(noise))) return OIC_EINVAL;
    OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
    oic_status s = OIC_OK;
    if (h->cfg.noise_mode == OIC_NOISE_PHILOX) {
        // inputs into the workspace, the step graph, outputs out of it
        const Layout& L = h->lay;
        const size_t n = h->cfg.n, m = h->cfg.m, l = h->cfg.l, H = h->cfg.H;
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.xref), X_ref, sizeof(float) * (H + 1) * n * m,
                                    cudaMemcpyDeviceToDevice, h->st));
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.uref), U_ref, sizeof(float) * l * m, cudaMemcpyDeviceToDevice,
                                    h->st));
        if (!run_step_graph(h))
            s = step_impl(h, h->at<float>(L.xref), h->at<float>(L.uref), h->at<float>(L.noise),
                          h->at<float>(L.uapp), h->at<float>(L.xnext));
        if (s == OIC_OK && U_applied)
            OIC_CUDA_OK(cudaMemcpyAsync(U_applied, h->at<float>(L.uapp), sizeof(float) * l * m,
                                        cudaMemcpyDeviceToDevice, h->st));
        if (s == OIC_OK && X_next)
            OIC_CUDA_OK(cudaMemcpyAsync(X_next, h->at<float>(L.xnext), sizeof(float) * n * m,
                                        cudaMemcpyDeviceToDevice, h->st));
    } else {
        s = step_impl(h, X_ref, U_ref, noise, U_applied, X_next);
    }
    OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
    return s;
}

oic_status oic_reset_host(oic_handle* h, const float* X0, const float* U_prev)
{
    if (!h || !X0 || !U_prev) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const size_t n = h->cfg.n, m = h->cfg.m, l = h->cfg.l;
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantX), X0, sizeof(float) * n * m,
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantU), U_prev, sizeof(float) * l * m,
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    OIC_CUDA_OK(cudaMemsetAsync(h->at<char>(h->lay.ctr), 0, sizeof(unsigned long long), h->st));
    h->plant_ready = true;
    return OIC_OK;
}

oic_status oic_solve_host(oic_handle* h, const float* X_k, const float* U_prev, const float* X_ref,
                          const float* U_ref, const float* noise, float* U_hat, float* X_hat)
{
    if (!h || !X_k || !U_prev || !X_ref || !U_ref || !U_hat) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const oic_config& c = h->cfg;
    if (c.noise_mode == OIC_NOISE_HOST && !noise) return OIC_EINVAL;
    if (X_hat && !h->full()) return OIC_EINVAL;
    const size_t n = c.n, m = c.m, l = c.l, H = c.H;
    const Layout& L = h->lay;
    OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.xk), X_k, sizeof(float) * n * m, cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.uprev), U_prev, sizeof(float) * l * m, cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.xref), X_ref, sizeof(float) * (H + 1) * n * m,
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.uref), U_ref, sizeof(float) * l * m, cudaMemcpyHostToDevice, h->st));
    if (c.noise_mode == OIC_NOISE_HOST)
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.noise), noise, sizeof(float) * h->noise_n,
                                    cudaMemcpyHostToDevice, h->st));
    oic_status s = solve_impl(h, h->at<float>(L.xk), h->at<float>(L.uprev), h->at<float>(L.xref),
                              h->at<float>(L.uref), h->at<float>(L.noise), h->at<float>(L.uhat),
                              X_hat ? h->at<float>(L.xhat) : nullptr);
    if (s != OIC_OK) return s;
    OIC_CUDA_OK(cudaMemcpyAsync(U_hat, h->at<float>(L.uhat), sizeof(float) * (H + 1) * l * m,
                                cudaMemcpyDeviceToHost, h->st));
    if (X_hat)
        OIC_CUDA_OK(cudaMemcpyAsync(X_hat, h->at<float>(L.xhat), sizeof(float) * (H + 1) * n * m,
                                    cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
    return read_status(h);
}

oic_status oic_step_host(oic_handle* h, const float* X_ref, const float* U_ref, const float* noise,
                         float* U_applied, float* X_next)
{
    if (!h || !X_ref || !U_ref) return OIC_EINVAL;
    if (!h->bound || !h->plant_ready) return OIC_ESTATE;
    const oic_config& c = h->cfg;
    if (c.noise_mode == OIC_NOISE_HOST && !noise) return OIC_EINVAL;
    const size_t n = c.n, m = c.m, l = c.l, H = c.H;
    const Layout& L = h->lay;
    OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.xref), X_ref, sizeof(float) * (H + 1) * n * m,
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.uref), U_ref, sizeof(float) * l * m, cudaMemcpyHostToDevice, h->st));
    if (c.noise_mode == OIC_NOISE_HOST)
        OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(L.noise), noise, sizeof(float) * h->noise_n,
                                    cudaMemcpyHostToDevice, h->st));
    oic_status s = OIC_OK;
    if (!run_step_graph(h))
        s = step_impl(h, h->at<float>(L.xref), h->at<float>(L.uref), h->at<float>(L.noise), h->at<float>(L.uapp),
                      h->at<float>(L.xnext));
    if (s != OIC_OK) return s;
    if (U_applied)
        OIC_CUDA_OK(cudaMemcpyAsync(U_applied, h->at<float>(L.uapp), sizeof(float) * l * m,
                                    cudaMemcpyDeviceToHost, h->st));
    if (X_next)
        OIC_CUDA_OK(cudaMemcpyAsync(X_next, h->at<float>(L.xnext), sizeof(float) * n * m,
                                    cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
    return read_status(h);
}

oic_status oic_cnn_forward(oic_handle* h, int batch, const float* X, const float* U, float* X_next)
{
    if (!h || !X || !U || !X_next || batch < 1 || batch > h->cfg.N) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const long nx = (long)h->cfg.n * h->cfg.m, nu = (long)h->cfg.l * h->cfg.m;
    // X_next must not overlap X: tiles of neighbouring rows read X rows that
    // another tile writes
    const float* xe = X + (size_t)batch * nx;
    const float* ye = X_next + (size_t)batch * nx;
    if (X_next < xe && X < ye) return OIC_EINVAL;
    cnn_forward(h, batch, X, nx, U, nu, X_next, nx);
    return last_cuda();
}

oic_status oic_enks_update(oic_handle* h, int R, const int* obs_rows, float* E, const float* V,
                           const float* Ybar)
{
    if (!h || !obs_rows || !E || !V || !Ybar) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    if (R < 1 || R > h->R_act_max) return OIC_EINVAL;
    if (!aligned16(E) || !aligned16(V)) return OIC_EINVAL;
    const int p = h->p - h->nc;                          // p_obs = n + l
    for (int c = 0; c < p; ++c)
        if (obs_rows[c] < 0 || obs_rows[c] >= R) return OIC_EINVAL;
    int* gen = h->act_rows(h->cfg.H + 1);
    int* gobs = gen + h->R_act_max;
    OIC_CUDA_OK(cudaMemcpyAsync(gobs, obs_rows, sizeof(int) * p, cudaMemcpyHostToDevice, h->st));
    RowSet act{gen, R};
    RowSet obs{gobs, p};
    const ObsNoise Vn = obs_noise_buf(V, V, p);
    analysis(h, E, (long)R * h->cfg.m, act, obs, Vn, Ybar, Ybar, p);
    return last_cuda();
}

oic_status oic_sync(oic_handle* h)
{
    if (!h) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    return read_status(h);
}

float oic_last_ms(oic_handle* h)
{
    if (!h || !h->ev0 || !h->ev1) return -1.f;
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) != cudaSuccess) return -1.f;
    return ms;
}

oic_status oic_profile_begin(oic_handle* h, unsigned stage_mask, int max_launches)
{
    if (!h || max_launches < 1) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    Profiler& P = h->prof;
    if ((int)P.ev.size() < 2 * max_launches) {
        for (cudaEvent_t e : P.ev) cudaEventDestroy(e);
        P.ev.assign(2 * (size_t)max_launches, nullptr);
        for (auto& e : P.ev) OIC_CUDA_OK(cudaEventCreate(&e));
        P.stage.assign(max_launches, 0);
    }
    P.max = max_launches;
    P.mask = stage_mask;
    P.used = 0;
    P.every = 1;
    P.phase = 0;
    P.on = true;
    return OIC_OK;
}

oic_status oic_profile_sample(oic_handle* h, int every, int phase)
{
    if (!h || every < 1 || phase < 0 || phase >= every) return OIC_EINVAL;
    if (!h->prof.on) return OIC_ESTATE;
    h->prof.every = every;
    h->prof.phase = phase;
    return OIC_OK;
}

oic_status oic_profile_end(oic_handle* h, float* ms, int* launches)
{
    if (!h || !ms || !launches) return OIC_EINVAL;
    Profiler& P = h->prof;
    for (int s = 0; s < OIC_NUM_STAGES; ++s) { ms[s] = 0.f; launches[s] = 0; }
    if (!P.on) return OIC_ESTATE;
    P.on = false;
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    for (int u = 0; u < P.used; ++u) {
        float t = 0.f;
        OIC_CUDA_OK(cudaEventElapsedTime(&t, P.ev[2 * u], P.ev[2 * u + 1]));
        ms[P.stage[u]] += t;
        launches[P.stage[u]] += 1;
    }
    return OIC_OK;
}

unsigned long long oic_launch_count(void) { return g_launches.load(); }

oic_status oic_get_plan(const oic_handle* h, oic_plan* plan, oic_plan* limits)
{
    if (!h || !plan) return OIC_EINVAL;
    *plan = effective_plan(h);
    if (limits) *limits = plan_limits(h);
    return OIC_OK;
}

oic_status oic_set_plan(oic_handle* h, const oic_plan* plan)
{
    if (!h || !plan) return OIC_EINVAL;
    const oic_plan l = plan_limits(h);
    if (plan->stats_splits < 0 || plan->stats_splits > l.stats_splits || plan->update_ctas < 0 ||
        plan->update_ctas > l.update_ctas || plan->cnn_ctas < 0 || plan->cnn_ctas > l.cnn_ctas)
        return OIC_EINVAL;
    h->plan = *plan;
    drop_step_graphs(h);
    return OIC_OK;
}

oic_status oic_autotune(oic_handle* h, int reps, int flags, oic_plan* chosen, float* ms_rule, float* ms_tuned)
{
    if (!h || reps < 1 || reps > 1000) return OIC_EINVAL;
    if (!h->bound || !h->plant_ready || h->prof.on) return OIC_ESTATE;
    if (ms_rule) *ms_rule = -1.f;
    if (ms_tuned) *ms_tuned = -1.f;
    const std::string key = plan_key(h);
    if (!(flags & OIC_TUNE_FORCE)) {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        const auto it = g_plan_cache.find(key);
        if (it != g_plan_cache.end()) {
            h->plan = it->second;
            drop_step_graphs(h);
            if (chosen) *chosen = effective_plan(h);
            return OIC_OK;
        }
    }
    // the state the tuning steps disturb, restored at the end
    std::vector<unsigned char> saved(oic_state_bytes(h));
    oic_status s = oic_save_state(h, saved.data());
    if (s != OIC_OK) return s;
    const oic_plan entry = h->plan;
    const oic_config& c = h->cfg;
    const Layout& L = h->lay;
    const size_t n = c.n, m = c.m, l = c.l, H = c.H;
    // inputs: zero references; device-drawn noise where the caller supplies it
    OIC_CUDA_OK(cudaMemsetAsync(h->at<float>(L.xref), 0, sizeof(float) * (H + 1) * n * m, h->st));
    OIC_CUDA_OK(cudaMemsetAsync(h->at<float>(L.uref), 0, sizeof(float) * l * m, h->st));
    if (c.noise_mode == OIC_NOISE_HOST) {
        const size_t N = c.N, e0 = N * l * m, e1 = e0 + H * N * l * m, e2 = e1 + H * N * n * m,
                     e3 = e2 + H * N * l * m, e4 = e3 + H * N * (size_t)h->nc * m;
        const size_t ends[5] = {e0, e1, e2, e3, e4};
        const float sig[5] = {(float)c.sigma_w, (float)c.sigma_w, (float)c.sigma_vx, (float)c.sigma_vu, h->c_sigma};
        launch_philox_noise(h->at<float>(L.noise), h->noise_n, c.seed, h->at<unsigned long long>(L.ctr), ends, sig,
                            h->nc > 0 ? 5 : 4, h->st);
    }
    auto one_step = [&]() -> oic_status {
        if (run_step_graph(h)) return last_cuda();
        return step_impl(h, h->at<float>(L.xref), h->at<float>(L.uref), h->at<float>(L.noise), h->at<float>(L.uapp),
                         h->at<float>(L.xnext));
    };
    auto time_plan = [&](const oic_plan& p, float* ms) -> oic_status {
        h->plan = p;
        drop_step_graphs(h);
        oic_status r = one_step();                  // untimed: captures the step graph
        for (int i = 0; i < reps && r == OIC_OK; ++i) {
            if (i == 0) OIC_CUDA_OK(cudaEventRecord(h->ev0, h->st));
            r = one_step();
        }
        if (r != OIC_OK) return r;
        OIC_CUDA_OK(cudaEventRecord(h->ev1, h->st));
        OIC_CUDA_OK(cudaEventSynchronize(h->ev1));
        float t = 0.f;
        OIC_CUDA_OK(cudaEventElapsedTime(&t, h->ev0, h->ev1));
        *ms = t / reps;
        return read_status(h);
    };
    oic_plan cur{};                                 // start from the rules
    float best = 0.f;
    s = time_plan(cur, &best);
    const float rule_ms = best;
    const oic_plan base = effective_plan(h);
    // candidates per field, one field at a time
    for (int field = 0; field < 3 && s == OIC_OK; ++field) {
        std::vector<int> cand;
        if (field == 0) {
            for (int d : {8, 7, 6, 4}) cand.push_back(h->n_sm * d / 8);
        } else if (field == 1) {
            const int r = base.stats_splits;
            for (int v : {r, r / 2, 2 * r / 3, 3 * r / 2, 2 * r, c.N / 8}) cand.push_back(v);
        } else {
            for (int v : {148, 111, 74, 37}) cand.push_back(v);
        }
        const oic_plan lim = plan_limits(h);
        const int lim_f = field == 0 ? lim.cnn_ctas : field == 1 ? lim.stats_splits : lim.update_ctas;
        const oic_plan eff = [&] { h->plan = cur; return effective_plan(h); }();
        const int cur_v = field == 0 ? eff.cnn_ctas : field == 1 ? eff.stats_splits : eff.update_ctas;
        std::vector<int> tried{cur_v};
        for (int v : cand) {
            if (v < 1 || v > lim_f || std::find(tried.begin(), tried.end(), v) != tried.end()) continue;
            tried.push_back(v);
            oic_plan trial = cur;
            (field == 0 ? trial.cnn_ctas : field == 1 ? trial.stats_splits : trial.update_ctas) = v;
            float t = 0.f;
            s = time_plan(trial, &t);
            if (s != OIC_OK) break;
            if (t < 0.99f * best) {
                best = t;
                cur = trial;
            }
        }
    }
    if (s != OIC_OK) {
        h->plan = entry;
        drop_step_graphs(h);
        oic_load_state(h, saved.data());
        cudaStreamSynchronize(h->st);
        return s;
    }
    h->plan = cur;
    drop_step_graphs(h);
    s = oic_load_state(h, saved.data());
    if (s != OIC_OK) return s;
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        g_plan_cache[key] = cur;
    }
    if (chosen) *chosen = effective_plan(h);
    if (ms_rule) *ms_rule = rule_ms;
    if (ms_tuned) *ms_tuned = best;
    return OIC_OK;
}

oic_status oic_selftest(oic_handle* h, int* result)
{
    if (!h || !result) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    int* d = h->at<int>(h->lay.selftest);
    OIC_CUDA_OK(cudaMemsetAsync(d, 0, 64, h->st));
    launch_tc_selftest(d, h->st);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    OIC_CUDA_OK(cudaGetLastError());
    OIC_CUDA_OK(cudaMemcpyAsync(result, d, 5 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    if (result[0] == -1) return OIC_ETIMEOUT;
    return result[0] == 0 ? OIC_OK : OIC_ECUDA;
}

// ------------------------------------------------------------- problem state
// Host layout: int32 header {n, m, l, 0}, uint64 solve index, X [n][m],
// U [l][m] (float32).
namespace {
constexpr size_t STATE_HDR = 4 * sizeof(int32_t) + sizeof(unsigned long long);
}

size_t oic_state_bytes(const oic_handle* h)
{
    if (!h) return 0;
    return STATE_HDR + sizeof(float) * ((size_t)h->cfg.n * h->cfg.m + (size_t)h->cfg.l * h->cfg.m);
}

oic_status oic_save_state(oic_handle* h, void* dst)
{
    if (!h || !dst) return OIC_EINVAL;
    if (!h->bound || !h->plant_ready) return OIC_ESTATE;
    const oic_config& c = h->cfg;
    char* d = static_cast<char*>(dst);
    const int32_t hdr[4] = {c.n, c.m, c.l, 0};
    std::memcpy(d, hdr, sizeof(hdr));
    OIC_CUDA_OK(cudaMemcpyAsync(d + sizeof(hdr), h->at<char>(h->lay.ctr), sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(d + STATE_HDR, h->at<float>(h->lay.plantX), sizeof(float) * c.n * c.m,
                                cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(d + STATE_HDR + sizeof(float) * c.n * c.m, h->at<float>(h->lay.plantU),
                                sizeof(float) * c.l * c.m, cudaMemcpyDeviceToHost, h->st));
    OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    return OIC_OK;
}

oic_status oic_load_state(oic_handle* h, const void* src)
{
    if (!h || !src) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const oic_config& c = h->cfg;
    const char* d = static_cast<const char*>(src);
    int32_t hdr[4];
    std::memcpy(hdr, d, sizeof(hdr));
    if (hdr[0] != c.n || hdr[1] != c.m || hdr[2] != c.l) return OIC_EINVAL;
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<char>(h->lay.ctr), d + sizeof(hdr), sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantX), d + STATE_HDR, sizeof(float) * c.n * c.m,
                                cudaMemcpyHostToDevice, h->st));
    OIC_CUDA_OK(cudaMemcpyAsync(h->at<float>(h->lay.plantU), d + STATE_HDR + sizeof(float) * c.n * c.m,
                                sizeof(float) * c.l * c.m, cudaMemcpyHostToDevice, h->st));
    h->plant_ready = true;
    return OIC_OK;
}

// ---------------------------------------------------------------- batching
struct oic_batch {
    std::vector<oic_handle*> hs;
    cudaStream_t st = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    unsigned long long launches = 0;
};

oic_status oic_io_slots(const oic_handle* h, float** X_ref, float** U_ref, float** U_applied, float** X_next)
{
    if (!h) return OIC_EINVAL;
    if (!h->bound) return OIC_ESTATE;
    const Layout& L = h->lay;
    if (X_ref) *X_ref = h->at<float>(L.xref);
    if (U_ref) *U_ref = h->at<float>(L.uref);
    if (U_applied) *U_applied = h->at<float>(L.uapp);
    if (X_next) *X_next = h->at<float>(L.xnext);
    return OIC_OK;
}

// (Re)captures one control step of every problem of b as one graph.
oic_status capture_batch(oic_batch* b)
{
    if (b->x) cudaGraphExecDestroy(b->x);
    if (b->g) cudaGraphDestroy(b->g);
    b->x = nullptr;
    b->g = nullptr;
    const int count = (int)b->hs.size();
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> join;
    try {
        br.assign(count, nullptr);
        join.assign(count, nullptr);
    } catch (...) {
        return OIC_ENOMEM;
    }
    // One capture: an origin stream forks to one stream per problem, each
    // problem's step is captured on its own stream (its kernels keep their
    // programmatic-dependency edges inside the branch), and the branches
    // join back.  The streams and events exist only during the capture.
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    bool ok = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < count; ++i)
        ok = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
    const unsigned long long l0 = g_launches.load();
    if (ok && cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        bool cap = cudaEventRecord(fork, origin) == cudaSuccess;
        for (int i = 0; cap && i < count; ++i) {
            oic_handle* h = b->hs[i];
            cap = cudaStreamWaitEvent(br[i], fork, 0) == cudaSuccess;
            StepGraph none;                       // capture mode, no profiling events
            const cudaStream_t own = h->st;
            h->st = br[i];
            h->capturing = &none;
            const Layout& L = h->lay;
            cap = cap && step_impl(h, h->at<float>(L.xref), h->at<float>(L.uref), h->at<float>(L.noise),
                                   h->at<float>(L.uapp), h->at<float>(L.xnext)) == OIC_OK;
            h->capturing = nullptr;
            h->st = own;
            cap = cap && cudaEventRecord(join[i], br[i]) == cudaSuccess &&
                  cudaStreamWaitEvent(origin, join[i], 0) == cudaSuccess;
        }
        cudaGraph_t g = nullptr;
        const bool ended = cudaStreamEndCapture(origin, &g) == cudaSuccess;
        b->g = g;
        ok = cap && ended && g != nullptr;
    } else {
        ok = false;
    }
    b->launches = g_launches.load() - l0;
    g_launches.fetch_sub(b->launches);                    // captured, not run
    ok = ok && cudaGraphInstantiate(&b->x, b->g, 0) == cudaSuccess;
    for (int i = 0; i < count; ++i) {
        if (join[i]) cudaEventDestroy(join[i]);
        if (br[i]) cudaStreamDestroy(br[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
    if (!ok) {
        cudaGetLastError();
        return OIC_ECUDA;
    }
    return OIC_OK;
}

oic_status oic_batch_create(oic_handle* const* handles, int count, void* cuda_stream, oic_batch** out)
{
    if (!handles || !out || count < 1 || count > 4096) return OIC_EINVAL;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        oic_handle* h = handles[i];
        if (!h) return OIC_EINVAL;
        if (h->cfg.noise_mode != OIC_NOISE_PHILOX) return OIC_EINVAL;
        if (!h->bound || !h->plant_ready) return OIC_ESTATE;
        for (int k = 0; k < i; ++k)
            if (handles[k] == h) return OIC_EINVAL;
    }
    oic_batch* b = new (std::nothrow) oic_batch;
    if (!b) return OIC_ENOMEM;
    try {
        b->hs.assign(handles, handles + count);
    } catch (...) {
        delete b;
        return OIC_ENOMEM;
    }
    b->st = static_cast<cudaStream_t>(cuda_stream);
    const oic_status s = capture_batch(b);
    if (s != OIC_OK) {
        oic_batch_destroy(b);
        return s;
    }
    *out = b;
    return OIC_OK;
}

oic_status oic_batch_autotune(oic_batch* b, int reps, float* ms_rule, float* ms_tuned)
{
    if (!b || reps < 1 || reps > 1000) return OIC_EINVAL;
    if (ms_rule) *ms_rule = -1.f;
    if (ms_tuned) *ms_tuned = -1.f;
    const int count = (int)b->hs.size();
    std::vector<std::vector<unsigned char>> saved(count);
    std::vector<oic_plan> entry(count);
    for (int i = 0; i < count; ++i) {
        oic_handle* h = b->hs[i];
        if (h->prof.on) return OIC_ESTATE;
        saved[i].resize(oic_state_bytes(h));
        const oic_status s = oic_save_state(h, saved[i].data());
        if (s != OIC_OK) return s;
        entry[i] = h->plan;
        const Layout& L = h->lay;
        OIC_CUDA_OK(cudaMemsetAsync(h->at<float>(L.xref), 0, sizeof(float) * (h->cfg.H + 1) * h->cfg.n * h->cfg.m,
                                    h->st));
        OIC_CUDA_OK(cudaMemsetAsync(h->at<float>(L.uref), 0, sizeof(float) * h->cfg.l * h->cfg.m, h->st));
        OIC_CUDA_OK(cudaStreamSynchronize(h->st));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OIC_CUDA_OK(cudaEventCreate(&e0));
    OIC_CUDA_OK(cudaEventCreate(&e1));
    // a choice applied to every problem: CNN CTAs as a fraction (eighths) of
    // the SMs, member-update CTAs, covariance splits as a fraction (eighths)
    // of each problem's rule
    struct Choice { int cnn8 = 8, upd = 0, split8 = 8; };
    auto apply = [&](const Choice& ch) {
        for (oic_handle* h : b->hs) {
            oic_plan p{};
            p.cnn_ctas = ch.cnn8 == 8 ? 0 : std::max(1, h->n_sm * ch.cnn8 / 8);
            p.update_ctas = ch.upd;
            p.stats_splits = ch.split8 == 8 ? 0 : std::max(1, rule_splits(h) * ch.split8 / 8);
            h->plan = p;
            drop_step_graphs(h);
        }
        return capture_batch(b);
    };
    auto time_choice = [&](const Choice& ch, float* ms) -> oic_status {
        oic_status s = apply(ch);
        if (s != OIC_OK) return s;
        OIC_CUDA_OK(cudaGraphLaunch(b->x, b->st));       // untimed
        OIC_CUDA_OK(cudaEventRecord(e0, b->st));
        for (int r = 0; r < reps; ++r) OIC_CUDA_OK(cudaGraphLaunch(b->x, b->st));
        OIC_CUDA_OK(cudaEventRecord(e1, b->st));
        OIC_CUDA_OK(cudaEventSynchronize(e1));
        float t = 0.f;
        OIC_CUDA_OK(cudaEventElapsedTime(&t, e0, e1));
        *ms = t / reps;
        for (oic_handle* h : b->hs) {
            s = read_status(h);
            if (s != OIC_OK) return s;
        }
        return OIC_OK;
    };
    Choice cur;
    float best = 0.f;
    oic_status s = time_choice(cur, &best);
    const float rule_ms = best;
    const int cnn_c[] = {6, 4, 2, 1}, upd_c[] = {74, 37, 18}, split_c[] = {4, 2};
    for (int field = 0; field < 3 && s == OIC_OK; ++field) {
        const int* cv = field == 0 ? cnn_c : field == 1 ? upd_c : split_c;
        const int nc = field == 0 ? 4 : field == 1 ? 3 : 2;
        for (int k = 0; k < nc && s == OIC_OK; ++k) {
            Choice trial = cur;
            (field == 0 ? trial.cnn8 : field == 1 ? trial.upd : trial.split8) = cv[k];
            float t = 0.f;
            s = time_choice(trial, &t);
            if (s == OIC_OK && t < 0.99f * best) {
                best = t;
                cur = trial;
            }
        }
    }
    if (s == OIC_OK) s = apply(cur);
    if (s != OIC_OK) {
        for (int i = 0; i < count; ++i) {
            b->hs[i]->plan = entry[i];
            drop_step_graphs(b->hs[i]);
        }
        capture_batch(b);
    }
    for (int i = 0; i < count; ++i) {
        const oic_status r = oic_load_state(b->hs[i], saved[i].data());
        if (s == OIC_OK) s = r;
        cudaStreamSynchronize(b->hs[i]->st);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != OIC_OK) return s;
    if (ms_rule) *ms_rule = rule_ms;
    if (ms_tuned) *ms_tuned = best;
    return OIC_OK;
}

oic_status oic_batch_step(oic_batch* b)
{
    if (!b || !b->x) return OIC_EINVAL;
    OIC_CUDA_OK(cudaGraphLaunch(b->x, b->st));
    g_launches.fetch_add(b->launches, std::memory_order_relaxed);
    return OIC_OK;
}

oic_status oic_batch_sync(oic_batch* b)
{
    if (!b) return OIC_EINVAL;
    OIC_CUDA_OK(cudaStreamSynchronize(b->st));
    oic_status first = OIC_OK;
    for (oic_handle* h : b->hs) {
        const oic_status s = read_status(h);
        if (first == OIC_OK) first = s;
    }
    return first;
}

void oic_batch_destroy(oic_batch* b)
{
    if (!b) return;
    if (b->x) cudaGraphExecDestroy(b->x);
    if (b->g) cudaGraphDestroy(b->g);
    delete b;
}

void oic_destroy(oic_handle* h)
{
    if (!h) return;
    for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    h->sg[0].reset();
    h->sg[1].reset();
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    delete h;
}

const char* oic_status_string(oic_status s)
{
    switch (s) {
    case OIC_OK: return "ok";
    case OIC_EINVAL: return "invalid argument";
    case OIC_ENOMEM: return "out of memory (workspace too small or host allocation failed)";
    case OIC_ECUDA: return "CUDA runtime error";
    case OIC_ENOTSPD: return "pseudo-observation covariance not positive definite";
    case OIC_ETIMEOUT: return "bounded device wait timed out";
    case OIC_ESTATE: return "call order violated (bind / reset first)";
    }
    return "unknown status";
}

const char* oic_version(void) { return "oic-b300 0.1 (sm_103a)"; }

}  // extern "C"
