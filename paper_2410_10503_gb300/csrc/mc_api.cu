// libmc host runtime: the C ABI of include/mc.h.
//
// Owns the per-context device state (tables, per-gate CSR of D_i^T, gated
// data, SPDHG/PDHG iterates, per-slot scratch), validates every call on the
// host, orders all work on the context's stream and replays whole epochs as
// CUDA graphs.  No computation of the method runs on the host: every step
// is one of the kernels in k_*.cu.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mc.h"
#include "mc_kernels.h"

using namespace mcg;

namespace {

std::mutex g_err_mu;
std::string g_create_err;

constexpr double kPi = 3.14159265358979323846;
constexpr int kPlanRounds = 6;   // re-cuts of the forward's items by simulated block time
constexpr int kNumClasses = 6;
const char* kClassNames[kNumClasses] = {"warp", "project", "backproject",
                                        "warp_adjoint_update", "gate_draw", "misc"};
enum { C_WARP = 0, C_PROJ = 1, C_BP = 2, C_WADJ = 3, C_DRAW = 4, C_MISC = 5 };

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};

struct Steps {
    double sigma = 0, tau = 0, theta = 0, kappa = 0, omega = 0;
};

void split_f(double v, float& hi, float& lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// v = hi + lo with hi rounded to 19 significant bits (so hi times any integer
// below 32 is exact in float32) and lo the float32 remainder.
void split_f19(double v, float& hi, float& lo)
{
    int e = 0;
    const double m = std::frexp(v, &e);                   // v = m 2^e, 0.5 <= |m| < 1
    const double h = std::ldexp(std::nearbyint(std::ldexp(m, 19)), e - 19);
    hi = (float)h;
    lo = (float)(v - h);
}

Steps make_steps(double norm2, double alpha, int N, double n_iter_per_epoch)
{
    // strongly convex PDHG/SPDHG steps: mu_g = 2 alpha, mu_f = N / 2
    Steps s;
    const double mu_g = 2.0 * alpha, mu_f = 0.5 * N;
    s.kappa = norm2 / (mu_g * mu_f);
    const double q = std::sqrt(1.0 + s.kappa);
    s.omega = 1.0 - 2.0 / ((double)n_iter_per_epoch * (1.0 + q));
    s.sigma = 1.0 / (mu_f * (q - 1.0));
    s.tau = (1.0 - s.omega) / (2.0 * mu_g * s.omega);
    s.theta = s.omega;
    return s;
}

}  // namespace

struct mc_ctx {
    int dev = 0, sms = 0;
    int n = 0, na = 0, nb = 0, N = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<void*> allocs;
    long fail_alloc_at = -1;          // simulated failure of the (k+1)-th device allocation

    // geometry
    FwdAngle* d_fang = nullptr;
    BpAngle* d_bang = nullptr;
    int2* d_groups = nullptr;
    RayItem* d_items = nullptr;
    int n_items = 0, ipb = 1, rpt = 1, lc = 1, P = 0, Gb = 0, Pb = 0, pj = 4;
    int guard = kGuardNarrow;         // zero pairs around each layout line (layout_guard)
    uint64_t tables_gen = 0;          // bumped whenever the forward tables or the launch
                                      // shapes change (batches made before refuse to run)
    size_t layout_stride = 0, dy_stride = 0;
    std::vector<int> order;           // angles, rows-driven first
    std::vector<double> inv_k, t_k;   // per angle: 1/|sin| or 1/|cos|, and the slope

    // sampling over gates x angle subsets: S subsets, blocks j = gate * S + s
    int S = 1;
    int2* d_sgroups = nullptr;
    RayItem* d_sitems = nullptr;
    int* d_soff = nullptr;
    int s_nitems = 0, s_ipb = 1, s_rpt = 2;
    int s_bands = 1;                  // line bands per subset item (partial sums in d_bandpart)
    float* d_bandpart = nullptr;
    int bands_opt = 0;                // MC_OPT_SUBSET_BANDS (0: min(8, max(1, S / 2)))
    int s_pj = 0;                     // MC_OPT_SUBSET_ROWS: backprojection rows per thread of the
                                      // subset launches (0: pj, the all-angle launches' height)

    // motion and D_i^T
    int kind = 0;
    RigidGate* d_rigid = nullptr;
    float* d_field = nullptr;
    int* d_rowptr = nullptr;
    int2* d_ent = nullptr;
    long long* d_ent_off = nullptr;
    int* d_csr_cnt = nullptr;     // per-row counters and scan scratch of a CSR rebuild
    int* d_csr_scan = nullptr;

    // data and iterates
    float* d_d = nullptr;
    float* d_y = nullptr;
    int store = 0;                    // MC_OPT_STORAGE: 0 float32 y (and d), 1 binary16, 2 bfloat16
    unsigned short* d_dh = nullptr;   // d and y in that storage type (d_d stays the float32 master)
    unsigned short* d_yh = nullptr;
    float* d_x[2] = {nullptr, nullptr};
    float* d_z = nullptr;
    int cur = 0;
    bool have_data = false;
    double alpha = 0;

    // staged upload of the next data set (mc_stage_data / mc_commit_data), allocated on first use
    float* d_stage = nullptr;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t stage_ev = nullptr;   // the staged upload has landed
    cudaEvent_t commit_ev = nullptr;  // the commit's device copy has read the staging buffer
    bool staged = false;

    // scratch per gate slot
    float2* d_lrow = nullptr;
    float2* d_lcol = nullptr;
    float2* d_dy = nullptr;
    float* d_b = nullptr;
    float* d_sinoN = nullptr;
    float* d_img[4] = {nullptr, nullptr, nullptr, nullptr};
    float* d_sino_io = nullptr;

    // control and reductions
    unsigned long long* d_k = nullptr;
    int* d_gates = nullptr;
    int gates_cap = 0;
    int* d_err = nullptr;
    int* h_err = nullptr;             // pinned copy of the error word for deferred checks
    cudaEvent_t err_ev = nullptr;     // that copy has landed
    bool err_pending = false;         // a deferred check is outstanding
    int* d_draw_out = nullptr;
    int draw_cap = 0;
    uint64_t k_host = 0;
    double* d_part = nullptr;
    double* d_s = nullptr;        // scalar slots
    double* d_trace = nullptr;
    int trace_cap = 0;

    // non-uniform serial sampling P(i) = p_i (mc_sampling.p): p normalised to
    // sum 1 (empty: uniform), the draw's thresholds and theta / p_i per gate as
    // uploaded (device tables allocated on first use)
    std::vector<double> p_steps;      // p the step sizes and coefficients follow
    std::vector<double> p_thr;        // p the uploaded thresholds follow
    std::vector<float> coef_host;     // theta / p_i as uploaded
    unsigned long long* d_thr = nullptr;
    float* d_coef = nullptr;

    // steps
    bool have_norms = false;
    std::vector<double> norms2;
    Steps sS, sP;
    bool steps_ok = false;

    // conjugate-gradient vectors (x, r, p, q), allocated on first use
    float* d_cg = nullptr;

    // reference
    float* d_xstar = nullptr;
    float* d_ystar = nullptr;
    bool have_ref = false;

    // options
    bool graph_on = true, prof_on = false, trace_obj = false;
    bool test_stall = false;          // MC_OPT_TEST_STALL: the next forward launch's waits run out

    // graphs: [0] SPDHG, [1] PDHG; index parity of cur at capture; which of the
    // two data buffers was current (commits swap d_d and d_stage)
    cudaGraphExec_t gexec[2][2][2] = {};
    int dsel = 0;
    uint64_t g_seed[2] = {0, 0};
    uint32_t g_stream[2] = {0, 0};

    // profiling
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    long long prof_count[kNumClasses] = {0};
    double prof_ms[kNumClasses] = {0};
};

// scalar slots in d_s
enum { S_DX2 = 0, S_XS2 = 1, S_DY2 = 2, S_XX = 3, S_TMP = 4, S_LAM = 5, S_NRM = 6,
       S_RR0 = 7, S_RR1 = 8, S_PQ = 9, S_BB = 10, S_RES = 16 };

namespace {

mc_status fail(mc_ctx* c, mc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
    } else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_err = buf;
    }
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, MC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#define TRY(expr)                       \
    do {                                \
        mc_status s_ = (expr);          \
        if (s_ != MC_OK) return s_;     \
    } while (0)

template <class T>
mc_status dalloc(mc_ctx* c, T** p, size_t count)
{
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (c->fail_alloc_at >= 0 && (long)c->allocs.size() >= c->fail_alloc_at)
        return fail(c, MC_ENOMEM, "simulated allocation failure at device buffer %zu (MC_FAIL_ALLOC_AFTER)",
                    c->allocs.size());
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, MC_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    e = cudaMemsetAsync(q, 0, bytes, c->stream);
    if (e != cudaSuccess) return fail(c, MC_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    *p = static_cast<T*>(q);
    return MC_OK;
}

// free one dalloc'd buffer early (stream work using it must have finished)
template <class T>
void dfree(mc_ctx* c, T** p)
{
    if (!*p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), (void*)*p);
    if (it != c->allocs.end()) {
        cudaFree(*it);
        c->allocs.erase(it);
    }
    *p = nullptr;
}

// 1 = device memory of this context's device, 0 = host, -1 = other device
int ptr_kind(mc_ctx* c, const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return (a.device == c->dev) ? 1 : -1;
    return 0;
}

mc_status check_ptr(mc_ctx* c, const void* p, const char* what)
{
    if (!p) return fail(c, MC_EINVAL, "%s is NULL", what);
    if (ptr_kind(c, p) < 0) return fail(c, MC_EINVAL, "%s lives on another device", what);
    return MC_OK;
}

cudaEvent_t ev_get(mc_ctx* c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;   // the launch then goes untimed
    }
    return e;
}

// launch through here: optional per-launch events for MC_OPT_PROFILE
template <class F>
mc_status launch(mc_ctx* c, int cls, const char* what, F&& f)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof_on) {
        a = ev_get(c);
        b = ev_get(c);
        if (!a || !b) {
            if (a) c->ev_pool.push_back(a);
            if (b) c->ev_pool.push_back(b);
            a = b = nullptr;
        }
    }
    if (a) cudaEventRecord(a, c->stream);
    const cudaError_t e = f();
    if (a) {
        cudaEventRecord(b, c->stream);
        c->prof.push_back({cls, a, b});
    }
    if (e != cudaSuccess) return fail(c, MC_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return MC_OK;
}

mc_status prof_collect(mc_ctx* c)
{
    if (c->prof.empty()) return MC_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (auto& r : c->prof) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->prof_count[r.cls] += 1;
            c->prof_ms[r.cls] += ms;
        } else {
            cudaGetLastError();
        }
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof.clear();
    return MC_OK;
}

mc_status check_err_word(mc_ctx* c)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h != kErrNone) {
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        if (h == kErrTimeout) return fail(c, MC_ETIMEOUT, "a device-side wait ran out of polls");
        return fail(c, MC_EDEVICE, "device error word %d (out-of-bounds sample)", h);
    }
    return MC_OK;
}

// Deferred check of the error word after a run that returns without waiting
// (device or no outputs): the word is copied to pinned host memory behind the
// run; poll_err reads it once that copy has landed (wait = false: only if it
// has, so a streaming caller is never held up) and reports a failure once.
mc_status defer_err(mc_ctx* c)
{
    if (!c->h_err) {
        void* p = nullptr;
        if (cudaHostAlloc(&p, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return check_err_word(c);     // no pinned word: check now
        }
        c->h_err = static_cast<int*>(p);
        *c->h_err = 0;
    }
    if (!c->err_ev) CK(cudaEventCreateWithFlags(&c->err_ev, cudaEventDisableTiming));
    CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaEventRecord(c->err_ev, c->stream));
    c->err_pending = true;
    return MC_OK;
}

mc_status poll_err(mc_ctx* c, bool wait)
{
    if (!c->err_pending) return MC_OK;
    if (wait) {
        CK(cudaEventSynchronize(c->err_ev));
    } else {
        const cudaError_t q = cudaEventQuery(c->err_ev);
        if (q == cudaErrorNotReady) return MC_OK;
        if (q != cudaSuccess) return fail(c, MC_ECUDA, "cudaEventQuery failed: %s", cudaGetErrorString(q));
    }
    c->err_pending = false;
    const int h = *c->h_err;
    if (h != kErrNone) {
        *c->h_err = kErrNone;
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
        if (h == kErrTimeout)
            return fail(c, MC_ETIMEOUT, "a device-side wait of an earlier run ran out of polls");
        return fail(c, MC_EDEVICE, "device error word %d of an earlier run (out-of-bounds sample)", h);
    }
    return MC_OK;
}

void drop_graphs(mc_ctx* c)
{
    for (auto& row : c->gexec)
        for (auto& pair : row)
            for (auto& g : pair)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

// ---- building blocks ------------------------------------------------------
mc_status warp_into_layouts(mc_ctx* c, const float* x, GateSel sel, int n_slots, bool identity)
{
    WarpArgs a{};
    a.x = x; a.n = c->n;
    a.rigid = c->d_rigid; a.field = c->d_field; a.identity = identity ? 1 : 0;
    a.sel = sel; a.n_slots = n_slots;
    a.lrow = c->d_lrow; a.lcol = c->d_lcol; a.layout_stride = c->layout_stride; a.P = c->P;
    a.guard = c->guard;
    return launch(c, C_WARP, "warp", [&] { return launch_warp_layouts(a, c->stream); });
}

FwdArgs fwd_args(mc_ctx* c, GateSel sel, int n_slots)
{
    FwdArgs a{};
    a.lrow = c->d_lrow; a.lcol = c->d_lcol; a.layout_stride = c->layout_stride; a.P = c->P;
    a.guard = c->guard;
    a.ang = c->d_fang; a.groups = c->d_groups; a.items = c->d_items; a.n_items = c->n_items;
    a.ipb = c->ipb; a.rpt = c->rpt; a.lc = c->lc; a.n = c->n; a.na = c->na; a.nb = c->nb;
    if (sel.subsets > 1) {            // the drawn block's angle subset
        a.groups = c->d_sgroups; a.items = c->d_sitems; a.sub_off = c->d_soff;
        a.n_items = c->s_nitems; a.ipb = c->s_ipb; a.rpt = c->s_rpt;
        if (c->s_bands > 1) {
            const int nch = layout_lines(c->n) / c->lc;
            a.nbands = c->s_bands;
            a.cpb = (nch + c->s_bands - 1) / c->s_bands;
            a.part = c->d_bandpart;
        }
    }
    a.sel = sel; a.n_slots = n_slots;
    a.wait_limit = 1u << 24;
    if (c->test_stall) {              // MC_OPT_TEST_STALL: this launch's waits run out
        a.stall = 1;
        a.wait_limit = 1u << 12;
        c->test_stall = false;
    }
    a.dy = c->d_dy; a.dy_stride = c->dy_stride; a.Pb = c->Pb; a.Gb = c->Gb;
    a.err = c->d_err;
    return a;
}

mc_status project_store(mc_ctx* c, GateSel sel, int n_slots, float* out)
{
    FwdArgs a = fwd_args(c, sel, n_slots);
    a.mode = 0; a.out = out;
    return launch(c, C_PROJ, "project", [&] { return launch_forward(a, c->stream); });
}

mc_status backproject(mc_ctx* c, GateSel sel, int n_slots, float* out)
{
    BpArgs a{};
    a.sel = sel;
    a.dy = c->d_dy; a.dy_stride = c->dy_stride; a.Pb = c->Pb; a.Gb = c->Gb;
    a.ang = c->d_bang; a.n = c->n; a.na = c->na; a.nb = c->nb; a.n_slots = n_slots;
    a.pj = (sel.subsets > 1 && c->s_pj) ? c->s_pj : c->pj;
    a.out = out; a.err = c->d_err;
    return launch(c, C_BP, "backproject", [&] { return launch_backproject(a, c->stream); });
}

WarpAdjArgs wadj_args(mc_ctx* c, GateSel sel, int n_slots, const float* b)
{
    WarpAdjArgs a{};
    a.n = c->n; a.rowptr = c->d_rowptr; a.ent = c->d_ent; a.ent_off = c->d_ent_off;
    a.sel = sel; a.n_slots = n_slots; a.b = b;
    return a;
}

mc_status pad_sinos(mc_ctx* c, const float* y, int n_slots)
{
    for (int s = 0; s < n_slots; ++s) {
        const float* ys = y + (size_t)s * c->na * c->nb;
        float2* dys = c->d_dy + (size_t)s * c->dy_stride;
        TRY(launch(c, C_MISC, "pad", [&] {
            return launch_pad_sino(ys, dys, c->d_bang, c->na, c->nb, c->Pb, c->Gb, c->stream);
        }));
    }
    return MC_OK;
}

mc_status reduce(mc_ctx* c, const float* a, const float* b, size_t len, int mode, double* out)
{
    return launch(c, C_MISC, "reduce", [&] {
        return launch_reduce(a, b, len, mode, c->d_part, out, c->stream);
    });
}

// A_i^* applied to N_slots sinograms (already padded in d_dy), summed, into out
mc_status adjoint_from_dy(mc_ctx* c, GateSel sel, int n_slots, float* out)
{
    TRY(backproject(c, sel, n_slots, c->d_b));
    WarpAdjArgs a = wadj_args(c, sel, n_slots, c->d_b);
    a.out = out;
    return launch(c, C_WADJ, "warp_adjoint", [&] { return launch_warp_adjoint_store(a, c->stream); });
}

// ---- one epoch --------------------------------------------------------------
mc_status enqueue_spdhg_epoch(mc_ctx* c, uint64_t seed, uint32_t stream)
{
    const int N = c->N, nblk = N * c->S;     // blocks: gates, or gates x angle subsets
    const bool nonuni = !c->p_steps.empty();
    TRY(launch(c, C_DRAW, "draw_gates", [&] {
        return launch_draw_gates(seed, stream, c->d_k, 0, nblk, nblk, nonuni ? c->d_thr : nullptr, c->d_gates,
                                 c->stream);
    }));
    const float sigma = (float)c->sS.sigma;
    const float inv_den = (float)(1.0 / (1.0 + c->sS.sigma * N / 2.0));
    for (int j = 0; j < nblk; ++j) {
        const GateSel sel{c->d_gates + j, -1, c->S};
        float* xin = c->d_x[c->cur];
        float* xout = c->d_x[c->cur ^ 1];
        TRY(warp_into_layouts(c, xin, sel, 1, false));
        FwdArgs fa = fwd_args(c, sel, 1);
        fa.mode = 1; fa.d = c->d_d; fa.y = c->d_y; fa.sigma = sigma; fa.inv_den = inv_den;
        fa.pf_rowptr = c->d_rowptr; fa.pf_ent = c->d_ent; fa.pf_ent_off = c->d_ent_off;   // gate's CSR into L2
        fa.store = c->store; fa.dh = c->d_dh; fa.yh = c->d_yh;
        TRY(launch(c, C_PROJ, "project", [&] { return launch_forward(fa, c->stream); }));
        TRY(backproject(c, sel, 1, c->d_b));
        WarpAdjArgs wa = wadj_args(c, sel, 1, c->d_b);
        wa.z = c->d_z; wa.x_in = xin; wa.x_out = xout;
        wa.coef = (float)(c->sS.theta * nblk);            // theta / p_j, p_j = 1/(N S)
        wa.coef_tab = nonuni ? c->d_coef : nullptr;       // theta / p_i, non-uniform p
        wa.tau = (float)c->sS.tau;
        wa.prox_scale = (float)(1.0 / (1.0 + 2.0 * c->sS.tau * c->alpha));
        TRY(launch(c, C_WADJ, "warp_adjoint_update", [&] {
            return launch_warp_adjoint_update(wa, c->stream);
        }));
        c->cur ^= 1;
    }
    return MC_OK;
}

mc_status enqueue_pdhg_iter(mc_ctx* c)
{
    const int N = c->N;
    const GateSel sel{nullptr, -1};
    float* xin = c->d_x[c->cur];
    float* xout = c->d_x[c->cur ^ 1];
    TRY(warp_into_layouts(c, xin, sel, N, false));
    FwdArgs fa = fwd_args(c, sel, N);
    fa.mode = 1; fa.d = c->d_d; fa.y = c->d_y;
    fa.store = c->store; fa.dh = c->d_dh; fa.yh = c->d_yh;
    fa.sigma = (float)c->sP.sigma;
    fa.inv_den = (float)(1.0 / (1.0 + c->sP.sigma * N / 2.0));
    TRY(launch(c, C_PROJ, "project", [&] { return launch_forward(fa, c->stream); }));
    TRY(backproject(c, sel, N, c->d_b));
    WarpAdjArgs wa = wadj_args(c, sel, N, c->d_b);
    wa.z = c->d_z; wa.x_in = xin; wa.x_out = xout;
    wa.coef = (float)c->sP.theta;                          // p_i = 1
    wa.tau = (float)c->sP.tau;
    wa.prox_scale = (float)(1.0 / (1.0 + 2.0 * c->sP.tau * c->alpha));
    TRY(launch(c, C_WADJ, "warp_adjoint_update", [&] { return launch_warp_adjoint_update(wa, c->stream); }));
    c->cur ^= 1;
    return MC_OK;
}

// Run one epoch of `which` (0 SPDHG, 1 PDHG), as a graph replay when enabled.
mc_status run_epoch(mc_ctx* c, int which, uint64_t seed, uint32_t stream)
{
    auto enqueue = [&]() -> mc_status {
        return which == 0 ? enqueue_spdhg_epoch(c, seed, stream) : enqueue_pdhg_iter(c);
    };
    const int flips = (which == 0) ? ((c->N * c->S) & 1) : 1;
    if (!c->graph_on || c->prof_on || c->test_stall) return enqueue();
    const int par = c->cur, ds = c->dsel;
    if (which == 0 && (c->g_seed[0] != seed || c->g_stream[0] != stream)) {
        bool any = false;
        for (auto& pair : c->gexec[0])
            for (auto& g : pair) any = any || g;
        if (any) drop_graphs(c);
    }
    if (!c->gexec[which][par][ds]) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        const mc_status st = enqueue();
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        c->cur = par;
        if (st != MC_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail(c, MC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return fail(c, MC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e2));
        c->gexec[which][par][ds] = ge;
        if (which == 0) { c->g_seed[0] = seed; c->g_stream[0] = stream; }
    }
    CK(cudaGraphLaunch(c->gexec[which][par][ds], c->stream));
    c->cur ^= flips;
    return MC_OK;
}

// trace entry e for the current state; x^K is the buffer that was the input
// of the last iteration
mc_status enqueue_trace(mc_ctx* c, int e)
{
    double* out = c->d_trace + 3 * (size_t)e;
    const float* xk = c->d_x[c->cur ^ 1];
    const size_t n2 = (size_t)c->n * c->n;
    if (c->have_ref) {
        const size_t cnt = (size_t)c->N * c->na * c->nb;
        const float* yk = c->d_y;
        if (c->store != 0) {           // the stored dual, widened to float32
            TRY(launch(c, C_MISC, "from_store", [&] {
                return launch_from_store(c->d_yh, c->d_sinoN, cnt, c->store, c->stream);
            }));
            yk = c->d_sinoN;
        }
        TRY(reduce(c, xk, c->d_xstar, n2, kRedDiffSq, c->d_s + S_DX2));
        TRY(reduce(c, yk, c->d_ystar, cnt, kRedDiffSq, c->d_s + S_DY2));
        TRY(launch(c, C_MISC, "trace", [&] {
            return launch_trace_combine(c->d_s + S_DX2, c->d_s + S_XS2, c->d_s + S_DY2, out, c->stream);
        }));
    } else {
        TRY(launch(c, C_MISC, "nan", [&] { return launch_fill_nan(out, 2, c->stream); }));
    }
    if (c->trace_obj) {
        // O(x) with all N forward projections at once
        const size_t ns = (size_t)c->na * c->nb;
        TRY(warp_into_layouts(c, xk, GateSel{nullptr, -1}, c->N, false));
        TRY(project_store(c, GateSel{nullptr, -1}, c->N, c->d_sinoN));
        for (int i = 0; i < c->N; ++i)
            TRY(reduce(c, c->d_sinoN + i * ns, c->d_d + i * ns, ns, kRedDiffSq, c->d_s + S_RES + i));
        TRY(reduce(c, xk, nullptr, n2, kRedSumSq, c->d_s + S_XX));
        TRY(launch(c, C_MISC, "objective", [&] {
            return launch_objective_combine(c->d_s + S_XX, c->d_s + S_RES, c->N, c->alpha, c->N,
                                            out + 2, c->stream);
        }));
    } else {
        TRY(launch(c, C_MISC, "nan", [&] { return launch_fill_nan(out + 2, 1, c->stream); }));
    }
    return MC_OK;
}

mc_status update_steps(mc_ctx* c)
{
    if (!c->have_norms || !c->have_data) {
        c->steps_ok = false;
        drop_graphs(c);
        return MC_OK;
    }
    const int nblk = c->N * c->S;
    double mx = 0;
    for (int i = 0; i < nblk; ++i) mx = std::max(mx, c->norms2[i]);
    if (!(mx > 0) || !(c->norms2[nblk] > 0)) {
        c->steps_ok = false;
        drop_graphs(c);
        return fail(c, MC_EINVAL, "operator norms must be positive");
    }
    // non-uniform p: the steps of the uniform rule with n = 1 / min_i p_i, so
    // that omega tau sigma ||A_i||^2 = min_j p_j <= p_i for every gate
    double n_eff = nblk;
    if (!c->p_steps.empty()) n_eff = 1.0 / *std::min_element(c->p_steps.begin(), c->p_steps.end());
    const Steps s = make_steps(mx, c->alpha, c->N, n_eff);
    const Steps p = make_steps(c->norms2[nblk], c->alpha, c->N, 1);
    // captured epochs bake the steps into their kernel arguments
    auto same = [](const Steps& a, const Steps& b) {
        return a.sigma == b.sigma && a.tau == b.tau && a.theta == b.theta;
    };
    if (!c->steps_ok || !same(s, c->sS) || !same(p, c->sP)) drop_graphs(c);
    c->sS = s;
    c->sP = p;
    c->steps_ok = true;
    if (!c->p_steps.empty()) {
        // theta / p_i per gate, uploaded when it changed (the graphs read it
        // at run time)
        std::vector<float> cf(c->N);
        for (int i = 0; i < c->N; ++i) cf[i] = (float)(s.theta / c->p_steps[i]);
        if (cf != c->coef_host) {
            if (!c->d_coef) TRY(dalloc(c, &c->d_coef, c->N));
            c->coef_host = cf;
            CK(cudaMemcpyAsync(c->d_coef, c->coef_host.data(), c->N * sizeof(float), cudaMemcpyHostToDevice,
                               c->stream));
        }
    }
    return MC_OK;
}

// The sampling's p (normalised), or an empty vector for uniform sampling.
mc_status read_p(mc_ctx* c, const mc_sampling* smp, std::vector<double>& p)
{
    p.clear();
    if (!smp || !smp->p) return MC_OK;
    if (c->S > 1) return fail(c, MC_EINVAL, "non-uniform sampling (p) is defined over gates only (subsets = 1)");
    if (ptr_kind(c, smp->p) != 0) return fail(c, MC_EINVAL, "sampling p must be host memory");
    double sum = 0.0;
    for (int i = 0; i < c->N; ++i) {
        const double v = smp->p[i];
        if (!(v > 0.0) || !std::isfinite(v)) return fail(c, MC_EINVAL, "sampling p[%d] must be finite and > 0", i);
        sum += v;                                   // in gate order
    }
    p.resize(c->N);
    for (int i = 0; i < c->N; ++i) p[i] = smp->p[i] / sum;
    return MC_OK;
}

// Upload the draw's thresholds for p (non-empty): thr[i] = floor(2^32 (p_0 + ... + p_i)),
// the running sum taken in gate order, thr[N-1] = 2^32.
mc_status set_thresholds(mc_ctx* c, const std::vector<double>& p)
{
    if (p.empty() || p == c->p_thr) return MC_OK;
    if (!c->d_thr) TRY(dalloc(c, &c->d_thr, c->N));
    std::vector<unsigned long long> th(c->N);
    double cum = 0.0;
    for (int i = 0; i < c->N; ++i) {
        cum += p[i];
        th[i] = (unsigned long long)std::floor(cum * 4294967296.0);
    }
    th[c->N - 1] = 4294967296ULL;
    CK(cudaMemcpy(c->d_thr, th.data(), c->N * sizeof(unsigned long long), cudaMemcpyHostToDevice));
    c->p_thr = p;
    return MC_OK;
}

// Make the context follow the sampling of a run: thresholds, step sizes and
// theta / p_i.  A change of p drops the captured epochs.
mc_status apply_sampling(mc_ctx* c, const mc_sampling* smp)
{
    std::vector<double> p;
    TRY(read_p(c, smp, p));
    if (p == c->p_steps) return MC_OK;
    TRY(set_thresholds(c, p));
    c->p_steps = p;
    c->coef_host.clear();
    drop_graphs(c);
    return update_steps(c);
}

// copy an input to device memory if it is a host pointer
mc_status stage_in(mc_ctx* c, const float* src, float* scratch, size_t count, const float** dev)
{
    if (ptr_kind(c, src) == 1) { *dev = src; return MC_OK; }
    CK(cudaMemcpyAsync(scratch, src, count * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    *dev = scratch;
    return MC_OK;
}

// write a device result to dst (host or device) and wait for host copies
mc_status stage_out(mc_ctx* c, float* dst, const float* dev, size_t count)
{
    if (ptr_kind(c, dst) == 1) {
        if (dst != dev)
            CK(cudaMemcpyAsync(dst, dev, count * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        return MC_OK;
    }
    CK(cudaMemcpyAsync(dst, dev, count * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MC_OK;
}

mc_status finish(mc_ctx* c)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, MC_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
#ifdef MC_CHECKED
    TRY(check_err_word(c));       // bounds checks of the checked build
#endif
    if (c->prof_on) TRY(prof_collect(c));
    return MC_OK;
}

mc_status check_gate(mc_ctx* c, int gate)
{
    if (gate < 0 || gate >= c->N) return fail(c, MC_EINVAL, "gate %d out of range [0, %d)", gate, c->N);
    return MC_OK;
}

// ---- creation ---------------------------------------------------------------
// Forward angle table for chunks of lc lines: slope split into float pairs and
// the exact integer/fraction split of the per-chunk advance lc * t.
std::vector<FwdAngle> fwd_angles(const mc_ctx* c, int lc)
{
    std::vector<FwdAngle> fa(c->na);
    for (int k = 0; k < c->na; ++k) {
        const bool xd = (c->na <= 4 * k) && (4 * k <= 3 * c->na);
        const double inv = c->inv_k[k], t = c->t_k[k];
        FwdAngle f{};
        split_f(inv, f.inv_hi, f.inv_lo);
        split_f(t, f.t_hi, f.t_lo);
        const double step = (double)lc * t;
        const double si = std::floor(step);
        f.step_int = (int)si;
        f.step_frac = (float)(step - si);
        if (f.step_frac >= 1.0f) { f.step_frac = 0.0f; f.step_int += 1; }
        f.delta = (float)std::fabs(inv);
        f.dir = xd ? 1 : 0;
        fa[k] = f;
    }
    return fa;
}

// Ray groups of the forward projector (up to 32 consecutive bins of one
// angle) for S interleaved angle subsets: subset s holds the angles k = s
// (mod S), rows-driven angles first; its groups are sets[s] = {first,
// first columns-driven, end}.  cum holds running work weights (a fixed
// setup cost per group plus its chunks, weighted by their load wavefronts).
struct GroupTable {
    std::vector<int2> groups;
    std::vector<long long> cum;
    std::vector<std::array<long long, 3>> sets;
};

void group_chunk_costs(const mc_ctx* c, int k, int b0, int lc, std::vector<float>& cost);
double load_wavefronts(const mc_ctx* c, int k);

// The ray groups of the context's angle order (c->order), S subsets after
// one another, each with its estimated cost in the forward at lc-line chunks.
void build_groups(const mc_ctx* c, int S, int lc, GroupTable& gt)
{
    const int na = c->na, nb = c->nb;
    const int gpa = (nb + 31) / 32;                        // groups per angle
    std::vector<float> cost;
    gt.groups.clear();
    gt.cum.assign(1, 0);
    gt.sets.clear();
    gt.groups.reserve((size_t)na * gpa);
    gt.cum.reserve((size_t)na * gpa + 1);
    for (int sub = 0; sub < S; ++sub) {
        std::array<long long, 3> set{(long long)gt.groups.size(), -1, 0};
        for (int k : c->order) {
            if (k % S != sub) continue;
            const bool xd = (na <= 4 * k) && (4 * k <= 3 * na);
            if (xd && set[1] < 0) set[1] = (long long)gt.groups.size();
            // measured block times on rigid512 fit chunks x (2.8 + wf) (R^2
            // 0.91), wf the wavefronts of a half-warp's 64-bit load
            const double wf = load_wavefronts(c, k);
            for (int g = 0; g < gpa; ++g) {
                // the work k_forward does for the group: all 32 lanes over every
                // chunk of the union of its rays' line ranges, each chunk
                // weighted by the shared-memory wavefronts of the angle's loads
                group_chunk_costs(c, k, g * 32, lc, cost);
                long long w = 64;
                for (float q : cost) w += q > 0.0f ? (long long)(32.0 * lc * (2.8 + wf)) : 0LL;
                gt.groups.push_back(make_int2(k, g * 32));
                gt.cum.push_back(gt.cum.back() + w);
            }
        }
        set[2] = (long long)gt.groups.size();
        if (set[1] < 0) set[1] = set[2];
        gt.sets.push_back(set);
    }
}

// Cut every set into about ipb * sms items of equal weight (each driving-axis
// class separately: an item streams one line layout); the smallest ipb whose
// items hold at most warps * rpt groups, rpt in {2, 4, 8}.  Items of set
// s are items[set_off[s] .. set_off[s+1]).
void partition_items(const GroupTable& gt, int sms, int ipb_start, int warps, std::vector<RayItem>& items,
                     std::vector<int>& set_off, int& ipb, int& rpt)
{
    const std::vector<long long>& cum = gt.cum;
    for (ipb = std::max(ipb_start, 1);; ++ipb) {
        const int target = ipb * sms;
        items.clear();
        set_off.assign(1, 0);
        long long max_groups = 0;
        for (const auto& set : gt.sets) {
            const double total = (double)(cum[set[2]] - cum[set[0]]);
            for (int cls = 0; cls < 2; ++cls) {
                const long long b0 = cls == 0 ? set[0] : set[1], b1 = cls == 0 ? set[1] : set[2];
                if (b1 <= b0) continue;
                const double w = (double)(cum[b1] - cum[b0]);
                const int cnt = std::max(1, (int)std::lround(target * w / total));
                long long st = b0;
                for (int i = 1; i <= cnt && st < b1; ++i) {
                    const long long goal = cum[b0] + (long long)std::llround(w * i / cnt);
                    long long e = std::lower_bound(cum.begin() + st + 1, cum.begin() + b1 + 1, goal) - cum.begin();
                    e = std::min(std::max(e, st + 1), b1);
                    if (i == cnt) e = b1;
                    items.push_back(RayItem{(int)st, (int)e, cls, 0});
                    max_groups = std::max(max_groups, e - st);
                    st = e;
                }
            }
            set_off.push_back((int)items.size());
        }
        rpt = 2;
        while (rpt < 8 && forward_groups_per_block(rpt, warps) < max_groups) rpt <<= 1;
        if (forward_groups_per_block(rpt, warps) >= max_groups) return;
    }
}

// Chunks of lc lines that group {k, b0} visits in k_forward: its rays cover
// lines [lo, hi] (the kernel's estimate, widened by one line on each side) and
// the group visits the union of their chunks, each at the same cost (one
// chunk of samples of all 32 lanes plus the per-chunk set-up of the group;
// measured per-block times follow these counts, whatever the angle).
void group_chunk_costs(const mc_ctx* c, int k, int b0, int lc, std::vector<float>& cost)
{
    const int n = c->n, nb = c->nb, nch = layout_lines(n) / lc;
    const double h = 0.5 * (n - 1), hb = 0.5 * (nb - 1);
    const double inv = c->inv_k[k], t = c->t_k[k];
    cost.assign(nch, 0.0f);
    int lo_min = n, hi_max = -1;
    for (int l = 0; l < 32; ++l) {
        const int b = std::min(b0 + l, nb - 1);
        const double G = c->guard;
        const double u0 = h * t + (b - hb) * inv + h + G;
        int lo = n, hi = -1;
        if (std::fabs(t) < 1e-6) {
            if (u0 > G - 2.0 && u0 < G + n + 1.0) { lo = 0; hi = n - 1; }
        } else {
            const double e1 = (u0 - (G + n)) / t, e3 = (u0 - (G - 1)) / t;
            const double llo = std::max(std::floor(std::min(e1, e3)) - 1.0, 0.0);
            const double lhi = std::min(std::ceil(std::max(e1, e3)) + 1.0, (double)(n - 1));
            if (llo <= lhi) { lo = (int)llo; hi = (int)lhi; }
        }
        lo_min = std::min(lo_min, lo); hi_max = std::max(hi_max, hi);
    }
    if (hi_max < lo_min) return;
    for (int ch = lo_min / lc; ch <= hi_max / lc; ++ch) cost[ch] = 1.0f;
}

// Deal the groups of every item to k_forward's consumer warps so that each
// warp gets about the same work in every stretch of chunks.  The kernel maps
// the p-th entry of an item to warp p % W, slot p / W; the ring lets warps
// drift apart by only kStages - 1 chunks, so a warp with more active groups
// than its neighbours over such a stretch holds the whole block back (a
// round-robin deal in angle/bin order left the busiest warp with ~1.5x the
// mean work), and a block takes about the sum over chunks of its busiest
// warp's load.  Greedy: loads smoothed over a window of 2 kStages - 1 chunks;
// groups by decreasing total cost, each to the warp where it raises that sum
// least (ties: the warp with the least total), any warp taking up to two
// groups more than an even share (at most 8); the
// item is then rewritten as W x L entries, L the most groups any warp got,
// with empty entries {-1, 0} that the kernel skips.  The groups array and the
// items' ranges are rebuilt; rpt becomes the smallest slot count >= L.  The
// order of groups changes no result: each group's rays are summed by one warp
// in line order either way.
// Wavefronts per 64-bit shared load of a half-warp for angle k's 16
// consecutive bins: about 1 + min(1, 15 (|inv| - 1)), one near the driving
// axis and two from ~20 degrees on.
double load_wavefronts(const mc_ctx* c, int k)
{
    return 1.0 + std::min(1.0, 15.0 * (std::fabs(c->inv_k[k]) - 1.0));
}

// Run body(i) for i in [0, count) on the host's cores (items of a plan are
// independent); the results do not depend on the number of threads.
template <class F>
void parallel_for(size_t count, F&& body)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nt = (unsigned)std::min<size_t>(hw, count);
    if (nt <= 1) {
        for (size_t i = 0; i < count; ++i) body(i);
        return;
    }
    std::atomic<size_t> next{0};
    std::vector<std::thread> pool;
    pool.reserve(nt);
    for (unsigned t = 0; t < nt; ++t)
        pool.emplace_back([&] {
            for (size_t i = next++; i < count; i = next++) body(i);
        });
    for (auto& th : pool) th.join();
}

void balance_items(const mc_ctx* c, int lc, std::vector<int2>& groups, std::vector<RayItem>& items, int& rpt,
                   std::vector<double>* item_time = nullptr)
{
    const int W = forward_warps(lc, forward_part_lines(lc, c->guard)), half = forward_ring(lc, c->P) - 1;
    const int nch = layout_lines(c->n) / lc;
    struct Deal {
        std::vector<std::vector<int>> lists;
        double T = 0.0;
    };
    std::vector<Deal> deals(items.size());
    parallel_for(items.size(), [&](size_t ii) {
        const RayItem& it = items[ii];
        std::vector<std::vector<float>> win;        // windowed cost per group of the item
        std::vector<float> cost, load, total, top, wsum;
        std::vector<int> idx;
        std::vector<std::vector<int>>& lists = deals[ii].lists;
        lists.assign(W, {});
        const int m = it.end - it.begin;
        win.assign(m, std::vector<float>(nch, 0.0f));
        total.assign(m, 0.0f);
        std::vector<int> g_lo(m, nch), g_hi(m, -1);  // window range of each group
        for (int g = 0; g < m; ++g) {
            const int2 grp = groups[it.begin + g];
            group_chunk_costs(c, grp.x, grp.y, lc, cost);
            for (int ch = 0; ch < nch; ++ch) {
                if (cost[ch] == 0.0f) continue;
                total[g] += cost[ch];
                const int q0 = std::max(0, ch - half), q1 = std::min(nch - 1, ch + half);
                g_lo[g] = std::min(g_lo[g], q0);
                g_hi[g] = std::max(g_hi[g], q1);
                for (int q = q0; q <= q1; ++q) win[g][q] += cost[ch];
            }
        }
        idx.resize(m);
        for (int g = 0; g < m; ++g) idx[g] = g;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return total[a] > total[b]; });
        const int cap = std::min(8, (m + W - 1) / W + 2);
        load.assign((size_t)W * nch, 0.0f);
        top.assign(nch, 0.0f);
        wsum.assign(W, 0.0f);
        for (int g : idx) {
            int best_w = -1;
            float best = 0.0f;
            for (int w = 0; w < W; ++w) {
                if ((int)lists[w].size() >= cap) continue;
                // outside the group's window its cost is zero and a warp's load
                // never exceeds the top: those chunks add nothing
                float rise = 0.0f;
                for (int ch = g_lo[g]; ch <= g_hi[g]; ++ch)
                    rise += std::max(0.0f, load[(size_t)w * nch + ch] + win[g][ch] - top[ch]);
                if (best_w < 0 || rise < best || (rise == best && wsum[w] < wsum[best_w])) {
                    best = rise;
                    best_w = w;
                }
            }
            lists[best_w].push_back(g);
            wsum[best_w] += total[g];
            for (int ch = g_lo[g]; ch <= g_hi[g]; ++ch) {
                float& l = load[(size_t)best_w * nch + ch];
                l += win[g][ch];
                top[ch] = std::max(top[ch], l);
            }
        }
        if (item_time) {
            // the block's time in a model of the ring: a warp may start chunk ch
            // once every warp has released chunk ch - stages; a group's chunk
            // costs 2.8 + its angle's load wavefronts (the fit of measured block
            // times), plus a fixed share per chunk
            const int S = half + 1;
            std::vector<double> R((size_t)W * nch, 0.0), done((size_t)W * nch, 0.0);
            for (int w = 0; w < W; ++w)
                for (int g : lists[w]) {
                    const int2 grp = groups[it.begin + g];
                    group_chunk_costs(c, grp.x, grp.y, lc, cost);
                    const double f = 2.8 + load_wavefronts(c, grp.x);
                    for (int ch = 0; ch < nch; ++ch) R[(size_t)w * nch + ch] += cost[ch] * f;
                }
            double T = 0.0;
            for (int ch = 0; ch < nch; ++ch) {
                double gate = 0.0;
                if (ch >= S)
                    for (int w = 0; w < W; ++w) gate = std::max(gate, done[(size_t)w * nch + ch - S]);
                for (int w = 0; w < W; ++w) {
                    const double prev = ch > 0 ? done[(size_t)w * nch + ch - 1] : 0.0;
                    done[(size_t)w * nch + ch] = std::max(prev, gate) + R[(size_t)w * nch + ch] + 0.5;
                    if (ch == nch - 1) T = std::max(T, done[(size_t)w * nch + ch]);
                }
            }
            deals[ii].T = T;
        }
    });
    std::vector<int2> out;
    out.reserve(groups.size() + items.size() * W);
    int most = 1;
    for (size_t ii = 0; ii < items.size(); ++ii) {
        RayItem& it = items[ii];
        const auto& lists = deals[ii].lists;
        int L = 0;
        for (const auto& l : lists) L = std::max(L, (int)l.size());
        most = std::max(most, L);
        if (item_time) item_time->push_back(deals[ii].T);
        const int begin = (int)out.size();
        for (int sl = 0; sl < L; ++sl)
            for (int w = 0; w < W; ++w)
                out.push_back(sl < (int)lists[w].size() ? groups[it.begin + lists[w][sl]] : make_int2(-1, 0));
        it.begin = begin;
        it.end = (int)out.size();
    }
    groups.swap(out);
    rpt = 2;
    while (rpt < most) rpt <<= 1;
}

// Cut the groups of gt into items (partition_items), deal every item to the
// warps (balance_items) and, for refine > 0 rounds, re-cut with each group's
// weight scaled by its item's simulated block time over the mean (the time
// model of balance_items), keeping the cut whose slowest block is fastest.
// On return gt.groups holds the dealt group entries and items their ranges.
void plan_forward(const mc_ctx* c, int lc, int sms, int ipb_start, int refine, GroupTable& gt,
                  std::vector<RayItem>& items, std::vector<int>& set_off, int& ipb, int& rpt)
{
    const std::vector<int2> base = gt.groups;
    std::vector<double> wts(base.size());
    for (size_t g = 0; g < base.size(); ++g) wts[g] = (double)(gt.cum[g + 1] - gt.cum[g]);
    double best_T = -1.0;
    std::vector<int2> best_groups;
    std::vector<RayItem> best_items;
    std::vector<int> best_off;
    int best_ipb = 1, best_rpt = 2;
    for (int round = 0; round <= refine; ++round) {
        GroupTable t = gt;
        t.groups = base;
        for (size_t g = 0; g < base.size(); ++g) t.cum[g + 1] = t.cum[g] + (long long)std::llround(wts[g]);
        std::vector<RayItem> its;
        std::vector<int> off;
        int ipb_r = 1, rpt_r = 2;
        partition_items(t, sms, ipb_start, forward_warps(lc, forward_part_lines(lc, c->guard)), its, off, ipb_r,
                        rpt_r);
        const std::vector<RayItem> cut = its;        // undealt ranges, for the re-weighting
        std::vector<double> T;
        balance_items(c, lc, t.groups, its, rpt_r, refine > 0 ? &T : nullptr);
        double Tmax = 0.0, Tsum = 0.0;
        for (double v : T) { Tmax = std::max(Tmax, v); Tsum += v; }
        if (best_T < 0.0 || Tmax < best_T) {
            best_T = Tmax;
            best_groups = t.groups;
            best_items = its;
            best_off = off;
            best_ipb = ipb_r;
            best_rpt = rpt_r;
        }
        if (refine == 0 || T.empty()) break;
        const double Tmean = Tsum / (double)T.size();
        for (size_t i = 0; i < cut.size(); ++i)
            for (int g = cut[i].begin; g < cut[i].end; ++g) wts[g] *= std::pow(T[i] / Tmean, 0.7);
    }
    gt.groups.swap(best_groups);
    items.swap(best_items);
    set_off.swap(best_off);
    ipb = best_ipb;
    rpt = best_rpt;
}

// The launch shapes and layout pitches a context of this geometry starts with
// (mc_create; mc_plan_shapes reports them without a device).
struct Shapes {
    int guard, P, lines, lc, cl, ring, pj, Gb, Pb;
};

Shapes choose_shapes(int n, int nb, int sms)
{
    Shapes sh{};
    // line layouts: `guard` zero pairs in front, >= guard behind, 16-byte
    // pitch, lines padded to whole chunks; chunks of lc in {16, 8, 4, 2} lines
    // per ring stage, the longest whose ring in the one block per SM keeps at
    // least 3 stages
    sh.guard = layout_guard(n);
    sh.P = layout_pitch(n, sh.guard);
    sh.lines = layout_lines(n);
    sh.lc = forward_default_lines(n, sh.P, sh.guard);
    sh.cl = forward_part_lines(sh.lc, sh.guard);
    sh.ring = forward_ring(sh.lc, sh.P);
    // backprojection tiles: 32 columns x pj rows per block of 8 warps.  Among
    // the tile heights whose grid still fills every SM's residency (4 blocks
    // of up to 16 rows, or 2 of 28: 24 and 16 warps per SM at least), the one
    // whose busiest SM does the least work: ceil(blocks / SMs) tiles, each
    // costing about 8 pj + 30 instructions per angle and lane (pj rows plus the
    // per-angle set-up), so that the grid fills whole waves (measured at
    // rigid512: 28 rows, 2 blocks per SM, ran the SPDHG epoch 4.6% faster than
    // 14 rows, 4 blocks per SM)
    sh.pj = 4;
    long long best_cost = -1;
    for (int pj : {28, 16, 14, 8}) {
        const long long blocks = (long long)((n + 31) / 32) * ((n + pj - 1) / pj);
        if (blocks < (pj > 16 ? 2LL : 3LL) * sms) continue;
        const long long cost = (blocks + sms - 1) / sms * (8LL * pj + 30);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; sh.pj = pj; }
    }
    // dual increment layout: guards wide enough for every pixel's two bins
    const double h = 0.5 * (n - 1), hb = 0.5 * (nb - 1);
    const int pj_max = 28;
    sh.Gb = std::max(2, (int)std::ceil(std::sqrt(2.0) * (h + pj_max + 1) - hb) + 2);
    sh.Pb = (nb + 2 * sh.Gb + 2 + 3) / 4 * 4;
    return sh;
}

mc_status build_tables(mc_ctx* c)
{
    const int n = c->n, na = c->na, nb = c->nb;
    const Shapes sh = choose_shapes(n, nb, c->sms);
    c->guard = sh.guard;
    c->P = sh.P;
    c->layout_stride = (size_t)sh.lines * c->P;
    c->lc = sh.lc;
    std::vector<FwdAngle> fa(na);
    std::vector<BpAngle> ba(na);
    // forward group order: rows-driven angles first, then columns-driven; in
    // each class the angles are taken round-robin from 8 contiguous bands, so
    // that every work item (a contiguous range of this order) mixes angles of
    // all obliquities -- long and short ray groups -- which lets the warp deal
    // of balance_items even out
    std::vector<int> order;
    order.reserve(na);
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int> cls;
        for (int k = 0; k < na; ++k) {
            const bool xd = (na <= 4 * k) && (4 * k <= 3 * na);
            if ((pass == 1) == xd) cls.push_back(k);
        }
        const int C = (int)cls.size(), B = (C + 7) / 8;
        for (int i = 0; i < B; ++i)
            for (int band = 0; band < 8; ++band)
                if (band * B + i < C) order.push_back(cls[band * B + i]);
    }
    std::vector<double> inv_k(na), t_k(na);
    for (int k = 0; k < na; ++k) {
        const double phi = (double)k * kPi / (double)na;
        const double cs = std::cos(phi), sn = std::sin(phi);
        const bool xd = (na <= 4 * k) && (4 * k <= 3 * na);
        const double inv = xd ? 1.0 / sn : 1.0 / cs;
        const double t = xd ? cs / sn : sn / cs;
        inv_k[k] = inv;
        t_k[k] = t;
        BpAngle b{};
        split_f(cs, b.cos_hi, b.cos_lo);
        split_f(sn, b.sin_hi, b.sin_lo);
        b.m = (float)std::fabs(inv);
        b.m2 = (float)(inv * inv);
        split_f19(cs, b.cos_h19, b.cos_l19);
        ba[k] = b;
    }
    // forward ray groups: up to 32 consecutive bins of one angle, rows-driven
    // angles first; work items cut each axis class into group ranges with
    // equal sample counts; one block per SM takes ipb consecutive items
    c->order = order;
    c->inv_k = inv_k;
    c->t_k = t_k;
    fa = fwd_angles(c, forward_part_lines(c->lc, c->guard));
    GroupTable gt;
    build_groups(c, 1, c->lc, gt);
    std::vector<RayItem> items;
    std::vector<int> set_off;
    int rpt = 2, ipb = 1;
    plan_forward(c, c->lc, c->sms, 1, kPlanRounds, gt, items, set_off, ipb, rpt);
    const std::vector<int2>& groups = gt.groups;
    c->ipb = ipb;
    c->rpt = rpt;
    c->n_items = (int)items.size();
    TRY(dalloc(c, &c->d_fang, na));
    TRY(dalloc(c, &c->d_bang, na));
    TRY(dalloc(c, &c->d_groups, groups.size()));
    TRY(dalloc(c, &c->d_items, items.size()));
    CK(cudaMemcpyAsync(c->d_fang, fa.data(), na * sizeof(FwdAngle), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_bang, ba.data(), na * sizeof(BpAngle), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_groups, groups.data(), groups.size() * sizeof(int2), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_items, items.data(), items.size() * sizeof(RayItem), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));   // host vectors go out of scope
    c->pj = sh.pj;
    c->Gb = sh.Gb;
    c->Pb = sh.Pb;
    c->dy_stride = (size_t)na * c->Pb;
    return MC_OK;
}

// Copy the dense field of gate g (2 x n x n floats at src + off, host or
// device) into the context and reject non-finite or absurd displacements
// (sample positions must stay below 2^22).
mc_status load_field(mc_ctx* c, int g, const float* src, size_t off)
{
    const size_t cnt = (size_t)2 * c->n * c->n;
    const int pk = ptr_kind(c, src);
    if (pk < 0) return fail(c, MC_EINVAL, "motion field lives on another device");
    std::vector<float> hf(cnt);
    if (pk == 1) {
        CK(cudaMemcpyAsync(hf.data(), src + off, cnt * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(hf.data(), src + off, cnt * sizeof(float));
    }
    for (size_t i = 0; i < cnt; ++i)
        if (!std::isfinite(hf[i]) || std::fabs(hf[i]) > 1.0e5f)
            return fail(c, MC_EINVAL, "motion field of gate %d, value %zu, is not finite or |u| > 1e5",
                        g, i);
    CK(cudaMemcpyAsync(c->d_field + (size_t)g * cnt, hf.data(), cnt * sizeof(float),
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return MC_OK;
}

mc_status build_motion(mc_ctx* c, const mc_motion* m)
{
    const int n = c->n, N = c->N;
    c->kind = m->kind;
    if (m->kind == MC_MOTION_RIGID) {
        std::vector<RigidGate> rg(N);
        const double h = 0.5 * (n - 1);
        for (int i = 0; i < N; ++i) {
            const double phi = m->rigid[3 * i], tx = m->rigid[3 * i + 1], ty = m->rigid[3 * i + 2];
            if (!std::isfinite(phi) || !std::isfinite(tx) || !std::isfinite(ty))
                return fail(c, MC_EINVAL, "rigid motion of gate %d is not finite", i);
            RigidGate g{};
            split_f(std::cos(phi), g.cos_hi, g.cos_lo);
            split_f(std::sin(phi), g.sin_hi, g.sin_lo);
            split_f(tx + h, g.offx_hi, g.offx_lo);
            split_f(ty + h, g.offy_hi, g.offy_lo);
            rg[i] = g;
        }
        TRY(dalloc(c, &c->d_rigid, N));
        CK(cudaMemcpyAsync(c->d_rigid, rg.data(), N * sizeof(RigidGate), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        TRY(dalloc(c, &c->d_field, (size_t)N * 2 * n * n));
        for (int g = 0; g < N; ++g) TRY(load_field(c, g, m->field, (size_t)g * 2 * n * n));
    }
    return MC_OK;
}

// CSR of D_g^T rebuilt in place.  Every pixel has at most four taps, so gate
// g owns a fixed slice of 4 n^2 entries (ent_off[g] = 4 n^2 g) and a rebuild
// after mc_set_field allocates nothing and moves no pointer.
mc_status build_gate_csr(mc_ctx* c, int g)
{
    const int n = c->n, n2 = n * n;
    const RigidGate* rg = c->d_rigid ? c->d_rigid + g : nullptr;
    const float* fl = c->d_field ? c->d_field + (size_t)g * 2 * n2 : nullptr;
    int* rp = c->d_rowptr + (size_t)g * (n2 + 1);
    int2* ent = c->d_ent + (size_t)g * 4 * n2;
    CK(cudaMemsetAsync(c->d_csr_cnt, 0, n2 * sizeof(int), c->stream));
    CK(launch_csr_count(n, rg, fl, c->d_csr_cnt, c->stream));
    CK(launch_exclusive_scan(c->d_csr_cnt, rp, n2, c->d_csr_scan, scan_scratch_len(n2), c->stream));
    CK(cudaMemsetAsync(c->d_csr_cnt, 0, n2 * sizeof(int), c->stream));
    CK(launch_csr_fill(n, rg, fl, rp, c->d_csr_cnt, ent, c->stream));
    CK(launch_csr_sort(n, rp, ent, c->stream));
    return MC_OK;
}

mc_status build_csr(mc_ctx* c)
{
    const int n = c->n, N = c->N, n2 = n * n;
    TRY(dalloc(c, &c->d_rowptr, (size_t)N * (n2 + 1)));
    TRY(dalloc(c, &c->d_ent, (size_t)N * 4 * n2));
    TRY(dalloc(c, &c->d_ent_off, N + 1));
    TRY(dalloc(c, &c->d_csr_cnt, n2));
    TRY(dalloc(c, &c->d_csr_scan, scan_scratch_len(n2)));
    std::vector<long long> off(N + 1);
    for (int g = 0; g <= N; ++g) off[g] = (long long)g * 4 * n2;
    CK(cudaMemcpyAsync(c->d_ent_off, off.data(), (N + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                       c->stream));
    for (int g = 0; g < N; ++g) TRY(build_gate_csr(c, g));
    CK(cudaStreamSynchronize(c->stream));
    return MC_OK;
}

mc_status alloc_state(mc_ctx* c)
{
    const size_t n2 = (size_t)c->n * c->n, ns = (size_t)c->na * c->nb;
    const int N = c->N;
    TRY(dalloc(c, &c->d_d, N * ns));
    TRY(dalloc(c, &c->d_y, N * ns));
    TRY(dalloc(c, &c->d_x[0], n2));
    TRY(dalloc(c, &c->d_x[1], n2));
    TRY(dalloc(c, &c->d_z, n2));
    TRY(dalloc(c, &c->d_lrow, N * c->layout_stride));
    TRY(dalloc(c, &c->d_lcol, N * c->layout_stride));
    TRY(dalloc(c, &c->d_dy, N * c->dy_stride));
    TRY(dalloc(c, &c->d_b, N * n2));
    TRY(dalloc(c, &c->d_sinoN, N * ns));
    for (auto& p : c->d_img) TRY(dalloc(c, &p, n2));
    TRY(dalloc(c, &c->d_sino_io, ns));
    TRY(dalloc(c, &c->d_k, 1));
    TRY(dalloc(c, &c->d_gates, std::max(N, 1)));
    c->gates_cap = std::max(N, 1);
    TRY(dalloc(c, &c->d_err, 1));
    TRY(dalloc(c, &c->d_part, reduce_parts()));
    TRY(dalloc(c, &c->d_s, S_RES + N + 8));
    return MC_OK;
}

}  // namespace

// ============================================================================
extern "C" {

const char* mc_version(void) { return "libmc 0.1 (sm_103a)"; }

mc_status mc_plan_shapes(const mc_geometry* geom, int32_t sms, int32_t* out)
{
    if (!geom || !out || sms < 1) return MC_EINVAL;
    if (geom->n < 2 || geom->n > 2048 || geom->n_angles < 1 || geom->n_angles > 8192 || geom->n_bins < 1 ||
        geom->n_bins > 8192)
        return MC_EINVAL;
    const Shapes sh = choose_shapes(geom->n, geom->n_bins, sms);
    const int32_t v[10] = {sh.guard, sh.P,  sh.lines, sh.lc, sh.cl, sh.ring,
                           sh.pj,    sh.Gb, sh.Pb,    forward_warps(sh.lc, sh.cl)};
    std::memcpy(out, v, sizeof v);
    return MC_OK;
}

mc_status mc_get_shapes(const mc_ctx* c, int32_t* out)
{
    if (!c || !out) return MC_EINVAL;
    const int cl = forward_part_lines(c->lc, c->guard);
    const int32_t v[10] = {c->guard, c->P,  layout_lines(c->n), c->lc, cl, forward_ring(c->lc, c->P),
                           c->pj,    c->Gb, c->Pb,              forward_warps(c->lc, cl)};
    std::memcpy(out, v, sizeof v);
    return MC_OK;
}

const char* mc_last_error(const mc_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    static thread_local std::string copy;
    copy = g_create_err;
    return copy.c_str();
}

void mc_destroy(mc_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (auto& r : c->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    if (c->commit_ev) cudaEventDestroy(c->commit_ev);
    if (c->err_ev) cudaEventDestroy(c->err_ev);
    if (c->h_err) cudaFreeHost(c->h_err);
    for (void* p : c->allocs) cudaFree(p);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

mc_status mc_create(const mc_geometry* geom, int32_t n_gates, const mc_motion* motion,
                    void* cuda_stream, mc_ctx** out)
{
    mc_ctx* c = nullptr;
    if (!out) return fail(nullptr, MC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!geom || !motion) return fail(nullptr, MC_EINVAL, "geometry or motion is NULL");
    if (geom->n < 2 || geom->n > 2048) return fail(nullptr, MC_EINVAL, "n=%d outside [2, 2048]", geom->n);
    if (geom->n_angles < 1 || geom->n_angles > 8192)
        return fail(nullptr, MC_EINVAL, "n_angles=%d outside [1, 8192]", geom->n_angles);
    if (geom->n_bins < 1 || geom->n_bins > 8192)
        return fail(nullptr, MC_EINVAL, "n_bins=%d outside [1, 8192]", geom->n_bins);
    if (n_gates < 1 || n_gates > 4096) return fail(nullptr, MC_EINVAL, "n_gates=%d outside [1, 4096]", n_gates);
    if (motion->kind == MC_MOTION_RIGID) {
        if (!motion->rigid) return fail(nullptr, MC_EINVAL, "rigid motion requires motion->rigid");
    } else if (motion->kind == MC_MOTION_FIELD) {
        if (!motion->field) return fail(nullptr, MC_EINVAL, "field motion requires motion->field");
    } else {
        return fail(nullptr, MC_EINVAL, "unknown motion kind %d", motion->kind);
    }
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(nullptr, MC_EDEVICE, "no CUDA device");
    }
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, MC_EDEVICE, "cudaGetDevice failed");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return fail(nullptr, MC_EDEVICE, "cudaGetDeviceProperties failed");
    if (prop.major * 10 + prop.minor != 103)
        return fail(nullptr, MC_EDEVICE, "libmc is built for sm_103a; device %d is sm_%d%d", dev,
                    prop.major, prop.minor);

    c = new (std::nothrow) mc_ctx();
    if (!c) return fail(nullptr, MC_ENOMEM, "host allocation failed");
    c->dev = dev;
    c->sms = prop.multiProcessorCount;
    if (const char* fa = std::getenv("MC_FAIL_ALLOC_AFTER")) c->fail_alloc_at = std::atol(fa);
    c->n = geom->n; c->na = geom->n_angles; c->nb = geom->n_bins; c->N = n_gates;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, MC_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    mc_status st = build_tables(c);
    if (st == MC_OK) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t static_smem = (size_t)forward_static_smem();   // per-warp group tables
        const size_t need = forward_smem_bytes(c->lc, c->P) + static_smem;
        if ((size_t)optin < need) st = fail(c, MC_EDEVICE, "forward needs %zu B shared memory", need);
        else if (forward_prepare(optin - (int)static_smem) != cudaSuccess || backproject_prepare() != cudaSuccess)
            st = fail(c, MC_ECUDA, "cudaFuncSetAttribute failed");
    }
    if (st == MC_OK) st = alloc_state(c);
    if (st == MC_OK) st = build_motion(c, motion);
    if (st == MC_OK) st = build_csr(c);
    if (st == MC_OK) {
        const cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = fail(c, MC_ECUDA, "setup failed: %s", cudaGetErrorString(e));
    }
    if (st != MC_OK) {
        fail(nullptr, st, "%s", c->err.c_str());
        mc_destroy(c);
        return st;
    }
    *out = c;
    return MC_OK;
}

mc_status mc_reset(mc_ctx* c)
{
    if (!c) return MC_EINVAL;
    const size_t n2 = (size_t)c->n * c->n, ns = (size_t)c->na * c->nb;
    // x^k, x^{k+1}, z, y (and its reduced-precision copy), the iteration counter: one launch
    ZeroSegs zs{};
    auto seg = [&](void* p, size_t bytes) { zs.ptr[zs.count] = p; zs.bytes[zs.count++] = bytes; };
    seg(c->d_x[0], n2 * sizeof(float));
    seg(c->d_x[1], n2 * sizeof(float));
    seg(c->d_z, n2 * sizeof(float));
    seg(c->d_y, (size_t)c->N * ns * sizeof(float));
    if (c->d_yh) seg(c->d_yh, (size_t)c->N * ns * sizeof(unsigned short));
    seg(c->d_k, sizeof(unsigned long long));
    TRY(launch(c, C_MISC, "reset", [&] { return launch_zero_segments(zs, c->stream); }));
    c->cur = 0;
    c->k_host = 0;
    return finish(c);
}

namespace {

// the part of mc_set_data after d has been copied into d_d on the context's
// stream; sync: wait for the stream (the caller's host array may be reused)
mc_status data_in_place(mc_ctx* c, double alpha, bool sync)
{
    const size_t cnt = (size_t)c->N * c->na * c->nb;
    if (c->store != 0)
        TRY(launch(c, C_MISC, "to_store", [&] { return launch_to_store(c->d_d, c->d_dh, cnt, c->store, c->stream); }));
    c->alpha = alpha;
    c->have_data = true;
    c->have_ref = false;
    TRY(mc_reset(c));
    TRY(update_steps(c));
    if (sync) CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

}  // namespace

mc_status mc_set_data(mc_ctx* c, const float* d, double alpha)
{
    if (!c) return MC_EINVAL;
    TRY(check_ptr(c, d, "d"));
    if (!(alpha > 0) || !std::isfinite(alpha)) return fail(c, MC_EINVAL, "alpha must be finite and > 0");
    const size_t cnt = (size_t)c->N * c->na * c->nb;
    CK(cudaMemcpyAsync(c->d_d, d, cnt * sizeof(float),
                       ptr_kind(c, d) == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return data_in_place(c, alpha, true);
}

mc_status mc_stage_data(mc_ctx* c, const float* d)
{
    if (!c) return MC_EINVAL;
    TRY(check_ptr(c, d, "d"));
    if (ptr_kind(c, d) != 0) return fail(c, MC_EINVAL, "d must be host memory (use mc_set_data for device data)");
    const size_t cnt = (size_t)c->N * c->na * c->nb;
    if (!c->d_stage) {
        TRY(dalloc(c, &c->d_stage, cnt));
        // dalloc clears the buffer on the context's stream: let that finish
        // before the copy stream writes into it
        CK(cudaStreamSynchronize(c->stream));
    }
    if (!c->copy_stream) CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    if (!c->stage_ev) CK(cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming));
    if (!c->commit_ev) CK(cudaEventCreateWithFlags(&c->commit_ev, cudaEventDisableTiming));
    // a commit still reading the staging buffer on the context's stream finishes first
    // (waiting on an event never recorded returns at once)
    CK(cudaStreamWaitEvent(c->copy_stream, c->commit_ev, 0));
    CK(cudaMemcpyAsync(c->d_stage, d, cnt * sizeof(float), cudaMemcpyHostToDevice, c->copy_stream));
    CK(cudaEventRecord(c->stage_ev, c->copy_stream));
    c->staged = true;
    return finish(c);
}

mc_status mc_commit_data(mc_ctx* c, double alpha)
{
    if (!c) return MC_EINVAL;
    if (!c->staged) return fail(c, MC_ESTATE, "no data staged (mc_stage_data)");
    if (!(alpha > 0) || !std::isfinite(alpha)) return fail(c, MC_EINVAL, "alpha must be finite and > 0");
    // the caller's host array is free once the upload has landed; the staged
    // buffer then becomes the data and the old data buffer the next staging
    // buffer (no device copy).  commit_ev marks the end of the work enqueued so
    // far, the last to read the old buffer: the next upload waits for it.
    CK(cudaEventSynchronize(c->stage_ev));
    CK(cudaEventRecord(c->commit_ev, c->stream));
    std::swap(c->d_d, c->d_stage);
    c->dsel ^= 1;
    c->staged = false;
    return data_in_place(c, alpha, false);
}

mc_status mc_forward(mc_ctx* c, int32_t gate, const float* x, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    TRY(check_ptr(c, x, "x"));
    TRY(check_ptr(c, out, "out"));
    const float* xd;
    TRY(stage_in(c, x, c->d_img[0], (size_t)c->n * c->n, &xd));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_sino_io;
    TRY(warp_into_layouts(c, xd, GateSel{nullptr, gate}, 1, false));
    TRY(project_store(c, GateSel{nullptr, gate}, 1, o));
    TRY(stage_out(c, out, o, (size_t)c->na * c->nb));
    return finish(c);
}

mc_status mc_project(mc_ctx* c, const float* x, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_ptr(c, x, "x"));
    TRY(check_ptr(c, out, "out"));
    const float* xd;
    TRY(stage_in(c, x, c->d_img[0], (size_t)c->n * c->n, &xd));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_sino_io;
    TRY(warp_into_layouts(c, xd, GateSel{nullptr, 0}, 1, true));
    TRY(project_store(c, GateSel{nullptr, 0}, 1, o));
    TRY(stage_out(c, out, o, (size_t)c->na * c->nb));
    return finish(c);
}

mc_status mc_adjoint(mc_ctx* c, int32_t gate, const float* y, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    TRY(check_ptr(c, y, "y"));
    TRY(check_ptr(c, out, "out"));
    const float* yd;
    TRY(stage_in(c, y, c->d_sino_io, (size_t)c->na * c->nb, &yd));
    TRY(pad_sinos(c, yd, 1));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_img[1];
    TRY(adjoint_from_dy(c, GateSel{nullptr, gate}, 1, o));
    TRY(stage_out(c, out, o, (size_t)c->n * c->n));
    return finish(c);
}

mc_status mc_backproject(mc_ctx* c, const float* y, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_ptr(c, y, "y"));
    TRY(check_ptr(c, out, "out"));
    const float* yd;
    TRY(stage_in(c, y, c->d_sino_io, (size_t)c->na * c->nb, &yd));
    TRY(pad_sinos(c, yd, 1));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_img[1];
    TRY(backproject(c, GateSel{nullptr, 0}, 1, o));
    TRY(stage_out(c, out, o, (size_t)c->n * c->n));
    return finish(c);
}

mc_status mc_warp(mc_ctx* c, int32_t gate, const float* x, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    TRY(check_ptr(c, x, "x"));
    TRY(check_ptr(c, out, "out"));
    const float* xd;
    TRY(stage_in(c, x, c->d_img[0], (size_t)c->n * c->n, &xd));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_img[1];
    WarpArgs a{};
    a.x = xd; a.n = c->n; a.rigid = c->d_rigid; a.field = c->d_field;
    a.sel = GateSel{nullptr, gate}; a.n_slots = 1; a.out = o;
    TRY(launch(c, C_WARP, "warp", [&] { return launch_warp_plain(a, c->stream); }));
    TRY(stage_out(c, out, o, (size_t)c->n * c->n));
    return finish(c);
}

mc_status mc_warp_adjoint(mc_ctx* c, int32_t gate, const float* v, float* out)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    TRY(check_ptr(c, v, "v"));
    TRY(check_ptr(c, out, "out"));
    const float* vd;
    TRY(stage_in(c, v, c->d_img[0], (size_t)c->n * c->n, &vd));
    const bool dev_out = ptr_kind(c, out) == 1;
    float* o = dev_out ? out : c->d_img[1];
    WarpAdjArgs a = wadj_args(c, GateSel{nullptr, gate}, 1, vd);
    a.out = o;
    TRY(launch(c, C_WADJ, "warp_adjoint", [&] { return launch_warp_adjoint_store(a, c->stream); }));
    TRY(stage_out(c, out, o, (size_t)c->n * c->n));
    return finish(c);
}

// Install the all-angle forward tables for chunks of lc lines and at least
// ipb_start items per block (rpt = 0: the smallest that fits, else at least rpt).
mc_status install_forward_tables(mc_ctx* c, int lc, int ipb_start, int rpt_min, int refine = 0)
{
    std::vector<FwdAngle> fa = fwd_angles(c, forward_part_lines(lc, c->guard));
    GroupTable gt;
    build_groups(c, 1, lc, gt);
    std::vector<RayItem> items;
    std::vector<int> off;
    int ipb = 1, rpt = 2;
    plan_forward(c, lc, c->sms, ipb_start, refine, gt, items, off, ipb, rpt);   // the deal depends on the cut and lc
    while (rpt < rpt_min && rpt < 8) rpt <<= 1;
    dfree(c, &c->d_items);
    dfree(c, &c->d_groups);
    TRY(dalloc(c, &c->d_items, items.size()));
    TRY(dalloc(c, &c->d_groups, gt.groups.size()));
    CK(cudaMemcpyAsync(c->d_fang, fa.data(), fa.size() * sizeof(FwdAngle), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_groups, gt.groups.data(), gt.groups.size() * sizeof(int2), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(c->d_items, items.data(), items.size() * sizeof(RayItem), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->lc = lc;
    c->ipb = ipb;
    c->rpt = rpt;
    c->n_items = (int)items.size();
    ++c->tables_gen;
    return MC_OK;
}

mc_status mc_autotune(mc_ctx* c, int32_t reps, int32_t* out)
{
    if (!c) return MC_EINVAL;
    if (reps < 1 || reps > 1000) return fail(c, MC_EINVAL, "reps must be in [1, 1000]");
    CK(cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        return fail(c, MC_ECUDA, "cudaEventCreate failed");
    }
    const bool prof = c->prof_on;
    c->prof_on = false;
    // each repetition timed on its own: launched back to back, a kernel's
    // successor (here the same kernel) would start in its tail and flatter
    // launch shapes whose tails the iteration's real successor does not hide
    auto timed = [&](auto&& body, float& ms) -> mc_status {
        TRY(body());                                   // warm-up
        ms = 0.0f;
        for (int r = 0; r < reps; ++r) {
            CK(cudaEventRecord(e0, c->stream));
            TRY(body());
            CK(cudaEventRecord(e1, c->stream));
            CK(cudaEventSynchronize(e1));
            float one = 0.0f;
            CK(cudaEventElapsedTime(&one, e0, e1));
            ms += one;
        }
        return MC_OK;
    };
    // the forward's work does not depend on the values: warp the current x of gate 0
    mc_status st = warp_into_layouts(c, c->d_x[c->cur], GateSel{nullptr, 0}, 1, false);
    // forward: chunk lines x items per block x group slots per warp
    int best_lc = c->lc, best_ipb = c->ipb, best_rpt = c->rpt;
    float best = 1e30f;
    for (int lc : {2, 4, 8, 16}) {
        if (st != MC_OK) break;
        if (!forward_lines_fit(c->n, c->P, c->guard, lc)) continue;   // guard, whole chunks, ring
        int ipb0 = 0;
        for (int step = 0; step < 3 && st == MC_OK; ++step) {
            const int ipb_try = ipb0 ? ipb0 + step : 1;
            for (int rmul = 1; rmul <= 2 && st == MC_OK; rmul *= 2) {
                st = install_forward_tables(c, lc, ipb_try, 0);
                if (st != MC_OK) break;
                if (!ipb0) ipb0 = c->ipb;
                if (rmul == 2) {
                    if (c->rpt >= 8) continue;
                    st = install_forward_tables(c, lc, ipb_try, c->rpt * 2);
                    if (st != MC_OK) break;
                }
                float ms = 0;
                st = timed([&] { return project_store(c, GateSel{nullptr, 0}, 1, c->d_sinoN); }, ms);
                if (st == MC_OK && ms < best) {
                    best = ms; best_lc = c->lc; best_ipb = c->ipb; best_rpt = c->rpt;
                }
            }
        }
    }
    if (st == MC_OK) st = install_forward_tables(c, best_lc, best_ipb, best_rpt, kPlanRounds);
    // backprojection: rows per thread, each candidate timed behind a forward
    // projection (as in the iteration, where the backprojection's blocks fill
    // the SMs as the forward's blocks drain); the forward is the same for all
    int best_pj = c->pj;
    float best_bp = 1e30f;
    for (int pj : {4, 8, 14, 16, 28}) {
        if (st != MC_OK) break;
        c->pj = pj;
        float ms = 0;
        st = timed([&] {
            TRY(project_store(c, GateSel{nullptr, 0}, 1, c->d_sinoN));
            return backproject(c, GateSel{nullptr, 0}, 1, c->d_b);
        }, ms);
        if (st == MC_OK && ms < best_bp) { best_bp = ms; best_pj = pj; }
    }
    c->pj = best_pj;
    ++c->tables_gen;
    // with angle subsets: the subset forward's line bands, its tables rebuilt
    // for each candidate and timed on the S blocks of gate 0 (forward, then
    // backprojection, block after block as in an epoch); norms and step sizes
    // are kept
    if (st == MC_OK && c->S > 1) {
        const bool had = c->have_norms;
        const std::vector<double> n2 = c->norms2;
        const int keep = c->bands_opt;
        int best_bands = keep;
        float best_sub = 1e30f;
        for (int bands : {1, 2, 3, 4, 6, 8}) {
            c->bands_opt = bands;
            st = mc_set_subsets(c, c->S);
            if (st != MC_OK) break;
            float ms = 0;
            st = timed([&]() -> mc_status {
                for (int j = 0; j < c->S; ++j) {
                    TRY(project_store(c, GateSel{nullptr, j, c->S}, 1, c->d_sinoN));
                    TRY(backproject(c, GateSel{nullptr, j, c->S}, 1, c->d_b));
                }
                return MC_OK;
            }, ms);
            if (st != MC_OK) break;
            if (ms < best_sub) { best_sub = ms; best_bands = bands; }
        }
        c->bands_opt = best_bands;
        const mc_status s2 = mc_set_subsets(c, c->S);
        if (st == MC_OK) st = s2;
        if (st == MC_OK && had) st = mc_set_norms(c, n2.data());
    }
    c->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(st);
    TRY(check_err_word(c));
    if (out) {
        out[0] = c->lc; out[1] = c->ipb; out[2] = c->rpt; out[3] = c->pj;
    }
    return finish(c);
}

mc_status mc_set_subsets(mc_ctx* c, int32_t subsets)
{
    if (!c) return MC_EINVAL;
    if (subsets < 1 || subsets > c->na)
        return fail(c, MC_EINVAL, "subsets must be in [1, n_angles = %d], got %d", c->na, subsets);
    CK(cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    dfree(c, &c->d_sgroups);
    dfree(c, &c->d_sitems);
    dfree(c, &c->d_soff);
    dfree(c, &c->d_bandpart);
    c->S = 1;
    c->s_bands = 1;
    c->have_norms = false;
    c->p_steps.clear();               // block sampling is uniform; a later run's p is applied anew
    c->coef_host.clear();
    if (subsets > 1) {
        // forward work items per angle subset, one table, subset s at soff[s];
        // with B = S / 2 line bands (at most 8) each subset's groups are cut
        // into ~SMs / B ranges, each repeated for every band
        const int bands = c->bands_opt > 0 ? c->bands_opt : std::min(8, std::max(1, subsets / 2));
        GroupTable gt;
        build_groups(c, subsets, c->lc, gt);
        std::vector<RayItem> cut;
        std::vector<int> cut_off;
        int ipb = 1, rpt = 2;
        partition_items(gt, std::max(1, c->sms / bands), 1, forward_warps(c->lc, forward_part_lines(c->lc, c->guard)),
                        cut, cut_off, ipb, rpt);
        balance_items(c, c->lc, gt.groups, cut, rpt);   // one deal serves every band of a cut
        std::vector<RayItem> items;
        std::vector<int> off(1, 0);
        for (int q = 0; q < subsets; ++q) {
            for (int band = 0; band < bands; ++band)
                for (int i = cut_off[q]; i < cut_off[q + 1]; ++i) {
                    RayItem it = cut[i];
                    it.band = band;
                    items.push_back(it);
                }
            off.push_back((int)items.size());
        }
        int most = 0;
        for (int q = 0; q < subsets; ++q) most = std::max(most, off[q + 1] - off[q]);
        if (bands > 1) TRY(dalloc(c, &c->d_bandpart, (size_t)bands * c->na * c->nb));
        c->s_bands = bands;
        TRY(dalloc(c, &c->d_sgroups, gt.groups.size()));
        TRY(dalloc(c, &c->d_sitems, items.size()));
        TRY(dalloc(c, &c->d_soff, off.size()));
        CK(cudaMemcpyAsync(c->d_sgroups, gt.groups.data(), gt.groups.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->d_sitems, items.data(), items.size() * sizeof(RayItem), cudaMemcpyHostToDevice,
                           c->stream));
        CK(cudaMemcpyAsync(c->d_soff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->s_nitems = most;
        c->s_ipb = ipb;
        c->s_rpt = rpt;
    }
    const int nblk = c->N * subsets;
    if (nblk > c->gates_cap) {
        dfree(c, &c->d_gates);
        TRY(dalloc(c, &c->d_gates, nblk));
        c->gates_cap = nblk;
    }
    c->S = subsets;
    TRY(update_steps(c));
    CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

mc_status mc_set_field(mc_ctx* c, int32_t gate, const float* field)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    if (c->kind != MC_MOTION_FIELD)
        return fail(c, MC_ESTATE, "mc_set_field needs a context created with dense-field motion");
    if (!field) return fail(c, MC_EINVAL, "field is NULL");
    TRY(load_field(c, gate, field, 0));
    TRY(build_gate_csr(c, gate));
    // A_gate changed: its norm, the step sizes and x* are stale
    c->have_norms = false;
    c->have_ref = false;
    TRY(update_steps(c));
    CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

mc_status mc_vjp(mc_ctx* c, int32_t gate, const float* x, const float* r, float* grad_x,
                 float* grad_field)
{
    if (!c) return MC_EINVAL;
    TRY(check_gate(c, gate));
    TRY(check_ptr(c, r, "r"));
    if (!grad_x && !grad_field) return fail(c, MC_EINVAL, "grad_x and grad_field are both NULL");
    if (grad_field) {
        if (c->kind != MC_MOTION_FIELD)
            return fail(c, MC_ESTATE, "grad_field needs a context created with dense-field motion");
        TRY(check_ptr(c, x, "x"));
        TRY(check_ptr(c, grad_field, "grad_field"));
    }
    if (grad_x) TRY(check_ptr(c, grad_x, "grad_x"));
    const size_t n2 = (size_t)c->n * c->n;
    const float* rd;
    TRY(stage_in(c, r, c->d_sino_io, (size_t)c->na * c->nb, &rd));
    TRY(pad_sinos(c, rd, 1));
    TRY(backproject(c, GateSel{nullptr, gate}, 1, c->d_b));     // b = A^T r
    if (grad_x) {
        const bool dev = ptr_kind(c, grad_x) == 1;
        float* o = dev ? grad_x : c->d_img[1];
        WarpAdjArgs a = wadj_args(c, GateSel{nullptr, gate}, 1, c->d_b);
        a.out = o;
        TRY(launch(c, C_WADJ, "warp_adjoint", [&] { return launch_warp_adjoint_store(a, c->stream); }));
        TRY(stage_out(c, grad_x, o, n2));
    }
    if (grad_field) {
        const float* xd;
        TRY(stage_in(c, x, c->d_img[0], n2, &xd));
        const bool dev = ptr_kind(c, grad_field) == 1;
        float* o0 = dev ? grad_field : c->d_img[2];
        float* o1 = dev ? grad_field + n2 : c->d_img[3];
        const float* fl = c->d_field + (size_t)gate * 2 * n2;
        TRY(launch(c, C_WARP, "field_vjp", [&] {
            return launch_field_vjp(c->n, fl, xd, c->d_b, o0, o1, c->stream);
        }));
        TRY(stage_out(c, grad_field, o0, n2));
        TRY(stage_out(c, grad_field + n2, o1, n2));
    }
    return finish(c);
}

mc_status mc_norms(mc_ctx* c, int32_t max_iter, double tol, double* out)
{
    if (!c) return MC_EINVAL;
    if (max_iter < 1 || !(tol >= 0)) return fail(c, MC_EINVAL, "max_iter >= 1 and tol >= 0 required");
    if (out && ptr_kind(c, out) < 0) return fail(c, MC_EINVAL, "out lives on another device");
    const size_t n2 = (size_t)c->n * c->n;
    float* v = c->d_img[2];
    float* w = c->d_img[3];
    const int nblk = c->N * c->S;
    std::vector<double> res(nblk + 1, 0.0);
    for (int which = 0; which <= nblk; ++which) {
        const bool stacked = which == nblk;
        const int slots = stacked ? c->N : 1;
        const GateSel sel = stacked ? GateSel{nullptr, -1} : GateSel{nullptr, which, c->S};
        // v = constant image of unit norm
        std::vector<float> ones(n2, (float)(1.0 / std::sqrt((double)n2)));
        CK(cudaMemcpyAsync(v, ones.data(), n2 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        double lam = 0;
        for (int it = 0; it < max_iter; ++it) {
            TRY(warp_into_layouts(c, v, sel, slots, false));
            TRY(project_store(c, sel, slots, c->d_sinoN));
            TRY(pad_sinos(c, c->d_sinoN, slots));
            TRY(adjoint_from_dy(c, sel, slots, w));
            TRY(reduce(c, v, w, n2, kRedDot, c->d_s + S_LAM));
            TRY(reduce(c, w, nullptr, n2, kRedSumSq, c->d_s + S_NRM));
            TRY(launch(c, C_MISC, "normalize", [&] { return launch_normalize(w, c->d_s + S_NRM, n2, c->stream); }));
            std::swap(v, w);
            double lam_new = 0;
            CK(cudaMemcpyAsync(&lam_new, c->d_s + S_LAM, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            const bool conv = lam > 0 && std::fabs(lam_new - lam) <= tol * lam_new;
            lam = lam_new;
            if (conv) break;
        }
        res[which] = lam;
    }
    c->norms2 = res;
    c->have_norms = true;
    TRY(update_steps(c));
    if (out) {
        if (ptr_kind(c, out) == 1)
            CK(cudaMemcpyAsync(out, res.data(), res.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        else
            std::memcpy(out, res.data(), res.size() * sizeof(double));
        CK(cudaStreamSynchronize(c->stream));
    }
    return finish(c);
}

mc_status mc_set_norms(mc_ctx* c, const double* norms2)
{
    if (!c) return MC_EINVAL;
    if (!norms2) return fail(c, MC_EINVAL, "norms2 is NULL");
    std::vector<double> v(c->N * c->S + 1);
    if (ptr_kind(c, norms2) == 1) {
        CK(cudaMemcpy(v.data(), norms2, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(v.data(), norms2, v.size() * sizeof(double));
    }
    for (double x : v)
        if (!(x > 0) || !std::isfinite(x)) return fail(c, MC_EINVAL, "norms must be finite and > 0");
    c->norms2 = v;
    c->have_norms = true;
    TRY(update_steps(c));
    return finish(c);
}

mc_status mc_get_steps(mc_ctx* c, int32_t pdhg, double* out)
{
    if (!c) return MC_EINVAL;
    if (!out) return fail(c, MC_EINVAL, "out is NULL");
    if (!c->steps_ok) return fail(c, MC_ESTATE, "step sizes need mc_set_data and mc_norms/mc_set_norms");
    const Steps& s = pdhg ? c->sP : c->sS;
    const double v[5] = {s.sigma, s.tau, s.theta, s.kappa, s.omega};
    std::memcpy(out, v, sizeof v);
    return MC_OK;
}

mc_status mc_set_reference(mc_ctx* c, const float* x_star)
{
    if (!c) return MC_EINVAL;
    if (!x_star) { c->have_ref = false; return MC_OK; }
    if (!c->have_data) return fail(c, MC_ESTATE, "mc_set_reference needs mc_set_data first");
    TRY(check_ptr(c, x_star, "x_star"));
    const size_t n2 = (size_t)c->n * c->n, ns = (size_t)c->na * c->nb;
    if (!c->d_xstar) {
        TRY(dalloc(c, &c->d_xstar, n2));
        TRY(dalloc(c, &c->d_ystar, (size_t)c->N * ns));
    }
    CK(cudaMemcpyAsync(c->d_xstar, x_star, n2 * sizeof(float),
                       ptr_kind(c, x_star) == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    TRY(reduce(c, c->d_xstar, nullptr, n2, kRedSumSq, c->d_s + S_XS2));
    // y_i* = (2/N)(A_i x* - d_i), all gates at once
    TRY(warp_into_layouts(c, c->d_xstar, GateSel{nullptr, -1}, c->N, false));
    TRY(project_store(c, GateSel{nullptr, -1}, c->N, c->d_ystar));
    const float s = (float)(2.0 / c->N);
    TRY(launch(c, C_MISC, "axpby", [&] {
        return launch_axpby(s, c->d_ystar, -s, c->d_d, c->d_ystar, (size_t)c->N * ns, c->stream);
    }));
    c->have_ref = true;
    CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

// (alpha I + N^-1 sum_i A_i^T A_i) v into out (all gates at once)
static mc_status apply_normal(mc_ctx* c, const float* v, float* out)
{
    const GateSel all{nullptr, -1};
    const size_t n2 = (size_t)c->n * c->n;
    TRY(warp_into_layouts(c, v, all, c->N, false));
    TRY(project_store(c, all, c->N, c->d_sinoN));
    TRY(pad_sinos(c, c->d_sinoN, c->N));
    TRY(adjoint_from_dy(c, all, c->N, out));
    const float inv_n = (float)(1.0 / c->N);
    const float al = (float)c->alpha;
    return launch(c, C_MISC, "axpby", [&] { return launch_axpby(al, v, inv_n, out, out, n2, c->stream); });
}

mc_status mc_solve_normal(mc_ctx* c, int32_t max_iter, double tol, float* x_out, double* info)
{
    if (!c) return MC_EINVAL;
    if (!c->have_data) return fail(c, MC_ESTATE, "mc_solve_normal needs mc_set_data first");
    if (max_iter < 1 || !(tol >= 0)) return fail(c, MC_EINVAL, "max_iter >= 1 and tol >= 0 required");
    TRY(check_ptr(c, x_out, "x_out"));
    const size_t n2 = (size_t)c->n * c->n;
    if (!c->d_cg) TRY(dalloc(c, &c->d_cg, 4 * n2));
    float *x = c->d_cg, *r = x + n2, *p = r + n2, *q = p + n2;
    CK(cudaMemsetAsync(x, 0, n2 * sizeof(float), c->stream));
    // r = p = b = N^-1 sum_i A_i^* d_i
    TRY(pad_sinos(c, c->d_d, c->N));
    TRY(adjoint_from_dy(c, GateSel{nullptr, -1}, c->N, r));
    const float inv_n = (float)(1.0 / c->N);
    TRY(launch(c, C_MISC, "axpby", [&] { return launch_axpby(inv_n, r, 0.0f, nullptr, r, n2, c->stream); }));
    CK(cudaMemcpyAsync(p, r, n2 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    TRY(reduce(c, r, nullptr, n2, kRedSumSq, c->d_s + S_BB));
    TRY(reduce(c, r, nullptr, n2, kRedSumSq, c->d_s + S_RR0));
    double bb = 0;
    CK(cudaMemcpyAsync(&bb, c->d_s + S_BB, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int it = 0;
    double rel = bb > 0 ? 1.0 : 0.0;
    double* rr = c->d_s + S_RR0;
    double* rr_new = c->d_s + S_RR1;
    while (it < max_iter && rel > tol) {
        TRY(apply_normal(c, p, q));
        TRY(reduce(c, p, q, n2, kRedDot, c->d_s + S_PQ));
        TRY(launch(c, C_MISC, "cg", [&] { return launch_cg_step1(x, r, p, q, n2, rr, c->d_s + S_PQ, c->stream); }));
        TRY(reduce(c, r, nullptr, n2, kRedSumSq, rr_new));
        TRY(launch(c, C_MISC, "cg", [&] { return launch_cg_step2(p, r, n2, rr_new, rr, c->stream); }));
        std::swap(rr, rr_new);
        ++it;
        if (it % 10 == 0 || it == max_iter) {
            double h = 0;
            CK(cudaMemcpyAsync(&h, rr, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            rel = bb > 0 ? std::sqrt(std::max(h, 0.0) / bb) : 0.0;
        }
    }
    TRY(stage_out(c, x_out, x, n2));
    if (info) { info[0] = it; info[1] = rel; }
    CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

static mc_status run_common(mc_ctx* c, int which, int32_t epochs, const mc_sampling* smp,
                            float* x_out, double* trace)
{
    if (!c) return MC_EINVAL;
    TRY(poll_err(c, false));              // a failure of an earlier run that did not wait
    if (epochs < 0) return fail(c, MC_EINVAL, "epochs must be >= 0");
    if (which == 0 && !smp) return fail(c, MC_EINVAL, "sampling is NULL");
    if (!c->have_data || !c->steps_ok)
        return fail(c, MC_ESTATE, "runs need mc_set_data and mc_norms/mc_set_norms first");
    if (x_out && ptr_kind(c, x_out) < 0) return fail(c, MC_EINVAL, "x_out lives on another device");
    if (trace && ptr_kind(c, trace) < 0) return fail(c, MC_EINVAL, "trace lives on another device");
    if (trace && epochs > c->trace_cap) {
        TRY(dalloc(c, &c->d_trace, 3 * (size_t)epochs));
        c->trace_cap = epochs;
    }
    if (which == 0) TRY(apply_sampling(c, smp));
    const uint64_t seed = smp ? smp->seed : 0;
    const uint32_t strm = smp ? smp->stream : 0;
    for (int e = 0; e < epochs; ++e) {
        TRY(run_epoch(c, which, seed, strm));
        if (which == 0) c->k_host += (uint64_t)c->N * c->S;
        if (trace) TRY(enqueue_trace(c, e));
    }
    if (x_out) TRY(stage_out(c, x_out, c->d_x[c->cur ^ 1], (size_t)c->n * c->n));
    if (trace && epochs > 0) {
        const bool dev = ptr_kind(c, trace) == 1;
        CK(cudaMemcpyAsync(trace, c->d_trace, 3 * (size_t)epochs * sizeof(double),
                           dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        if (!dev) CK(cudaStreamSynchronize(c->stream));
    }
    if (c->prof_on) TRY(prof_collect(c));
    const bool host_out = (x_out && ptr_kind(c, x_out) == 0) || (trace && ptr_kind(c, trace) == 0);
    if (!host_out) {
        // device or no outputs: return without waiting; the error word is
        // checked by a later run or by mc_sync
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(c, MC_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
        return defer_err(c);
    }
    TRY(poll_err(c, true));
    TRY(check_err_word(c));
    return finish(c);
}

mc_status mc_spdhg_run(mc_ctx* c, int32_t epochs, const mc_sampling* sampling, float* x_out,
                       double* trace)
{
    return run_common(c, 0, epochs, sampling, x_out, trace);
}

mc_status mc_batch_spdhg_run(mc_ctx* const* ctxs, int32_t count, int32_t epochs,
                             const mc_sampling* sampling, int32_t* failed)
{
    if (failed) *failed = -1;
    if (!ctxs || count < 1) return MC_EINVAL;
    if (!sampling) return fail(ctxs[0], MC_EINVAL, "sampling is NULL");
    if (epochs < 0) return fail(ctxs[0], MC_EINVAL, "epochs must be >= 0");
    int dev = -1;
    for (int i = 0; i < count; ++i) {
        mc_ctx* c = ctxs[i];
        if (!c) { if (failed) *failed = i; return MC_EINVAL; }
        if (i == 0) dev = c->dev;
        if (c->dev != dev || !c->have_data || !c->steps_ok) {
            if (failed) *failed = i;
            return fail(c, c->dev != dev ? MC_EINVAL : MC_ESTATE,
                        c->dev != dev ? "batch contexts must share one device"
                                      : "runs need mc_set_data and mc_norms/mc_set_norms first");
        }
        const mc_status st = apply_sampling(c, &sampling[i]);
        if (st != MC_OK) { if (failed) *failed = i; return st; }
    }
    // epoch by epoch, every slice in turn: each context's graph goes to its
    // own stream, so the slices' kernels overlap on the device
    for (int e = 0; e < epochs; ++e)
        for (int i = 0; i < count; ++i) {
            mc_ctx* c = ctxs[i];
            const mc_status st = run_epoch(c, 0, sampling[i].seed, sampling[i].stream);
            if (st != MC_OK) { if (failed) *failed = i; return st; }
            c->k_host += (uint64_t)c->N * c->S;
        }
    for (int i = 0; i < count; ++i) {
        mc_ctx* c = ctxs[i];
        mc_status st = check_err_word(c);
        if (st == MC_OK) st = finish(c);
        if (st != MC_OK) { if (failed) *failed = i; return st; }
    }
    return MC_OK;
}

mc_status mc_pdhg_run(mc_ctx* c, int32_t epochs, float* x_out, double* trace)
{
    return run_common(c, 1, epochs, nullptr, x_out, trace);
}

mc_status mc_draw_gates(mc_ctx* c, const mc_sampling* smp, uint64_t k0, int32_t count, int32_t* out)
{
    if (!c) return MC_EINVAL;
    if (!smp) return fail(c, MC_EINVAL, "sampling is NULL");
    if (count < 0) return fail(c, MC_EINVAL, "count must be >= 0");
    if (count == 0) return MC_OK;
    TRY(check_ptr(c, out, "out"));
    const bool dev = ptr_kind(c, out) == 1;
    int* o = out;
    if (!dev) {
        if (count > c->draw_cap) {
            TRY(dalloc(c, &c->d_draw_out, (size_t)count));
            c->draw_cap = count;
        }
        o = c->d_draw_out;
    }
    std::vector<double> p;
    TRY(read_p(c, smp, p));
    TRY(set_thresholds(c, p));
    TRY(launch(c, C_DRAW, "draw_gates", [&] {
        return launch_draw_gates(smp->seed, smp->stream, nullptr, k0, count, c->N * c->S,
                                 p.empty() ? nullptr : c->d_thr, o, c->stream);
    }));
    if (!dev) {
        CK(cudaMemcpyAsync(out, o, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return finish(c);
}

mc_status mc_objective(mc_ctx* c, const float* x, double* out)
{
    if (!c) return MC_EINVAL;
    if (!c->have_data) return fail(c, MC_ESTATE, "mc_objective needs mc_set_data first");
    TRY(check_ptr(c, x, "x"));
    if (!out) return fail(c, MC_EINVAL, "out is NULL");
    const size_t n2 = (size_t)c->n * c->n, ns = (size_t)c->na * c->nb;
    const float* xd;
    TRY(stage_in(c, x, c->d_img[0], n2, &xd));
    TRY(warp_into_layouts(c, xd, GateSel{nullptr, -1}, c->N, false));
    TRY(project_store(c, GateSel{nullptr, -1}, c->N, c->d_sinoN));
    for (int i = 0; i < c->N; ++i)
        TRY(reduce(c, c->d_sinoN + i * ns, c->d_d + i * ns, ns, kRedDiffSq, c->d_s + S_RES + i));
    TRY(reduce(c, xd, nullptr, n2, kRedSumSq, c->d_s + S_XX));
    TRY(launch(c, C_MISC, "objective", [&] {
        return launch_objective_combine(c->d_s + S_XX, c->d_s + S_RES, c->N, c->alpha, c->N,
                                        c->d_s + S_TMP, c->stream);
    }));
    double v = 0;
    CK(cudaMemcpyAsync(&v, c->d_s + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (ptr_kind(c, out) == 1) CK(cudaMemcpy(out, &v, sizeof v, cudaMemcpyHostToDevice));
    else *out = v;
    return finish(c);
}

mc_status mc_set_option(mc_ctx* c, int32_t option, int64_t value)
{
    if (!c) return MC_EINVAL;
    switch (option) {
    case MC_OPT_GRAPH: c->graph_on = value != 0; if (!c->graph_on) drop_graphs(c); return MC_OK;
    case MC_OPT_PROFILE: c->prof_on = value != 0; return MC_OK;
    case MC_OPT_TRACE_OBJECTIVE: c->trace_obj = value != 0; return MC_OK;
    case MC_OPT_TEST_STALL: c->test_stall = value != 0; return MC_OK;
    case MC_OPT_SUBSET_BANDS: {
        if (value < 0 || value > 8) return fail(c, MC_EINVAL, "subset bands must be in [0, 8]");
        c->bands_opt = (int)value;
        if (c->S <= 1) return MC_OK;
        // rebuild the subset tables with the new band count (norms and step sizes kept)
        const bool norms = c->have_norms;
        const std::vector<double> n2 = c->norms2;
        TRY(mc_set_subsets(c, c->S));
        if (norms) TRY(mc_set_norms(c, n2.data()));
        return MC_OK;
    }
    case MC_OPT_FORWARD_LINES: {
        const int lc = (int)value;
        if (lc != 2 && lc != 4 && lc != 8 && lc != 16)
            return fail(c, MC_EINVAL, "forward lines per chunk must be 2, 4, 8 or 16");
        if (!forward_lines_fit(c->n, c->P, c->guard, lc))
            return fail(c, MC_EINVAL, "chunks of %d lines do not fit this context's layouts (n = %d: room for "
                                      "%d ring stages, %d lines)", lc, c->n, forward_stages(lc, c->P),
                        layout_lines(c->n));
        CK(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        TRY(install_forward_tables(c, lc, 1, 0, kPlanRounds));
        if (c->S > 1) {               // the subset tables follow the chunk size
            const bool norms = c->have_norms;
            const std::vector<double> n2 = c->norms2;
            TRY(mc_set_subsets(c, c->S));
            if (norms) TRY(mc_set_norms(c, n2.data()));
        }
        return finish(c);
    }
    case MC_OPT_BACKPROJECT_ROWS:
        if (value != 4 && value != 8 && value != 14 && value != 16 && value != 28)
            return fail(c, MC_EINVAL, "backprojection rows per thread must be 4, 8, 14, 16 or 28");
        CK(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->pj = (int)value;
        ++c->tables_gen;
        return MC_OK;
    case MC_OPT_SUBSET_ROWS:
        if (value != 0 && value != 4 && value != 8 && value != 14 && value != 16 && value != 28)
            return fail(c, MC_EINVAL, "subset rows per thread must be 0, 4, 8, 14, 16 or 28");
        CK(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->s_pj = (int)value;
        return MC_OK;
    case MC_OPT_STORAGE: {
        if (value < 0 || value > 2) return fail(c, MC_EINVAL, "storage must be 0 (f32), 1 (f16) or 2 (bf16)");
        const int v = (int)value;
        if (v == c->store) return MC_OK;
        const size_t cnt = (size_t)c->N * c->na * c->nb;
        CK(cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        // carry the dual over: to float32 first, then to the new type
        if (c->store != 0)
            TRY(launch(c, C_MISC, "from_store", [&] {
                return launch_from_store(c->d_yh, c->d_y, cnt, c->store, c->stream);
            }));
        if (v != 0) {
            if (!c->d_yh) TRY(dalloc(c, &c->d_yh, cnt));
            if (!c->d_dh) TRY(dalloc(c, &c->d_dh, cnt));
            TRY(launch(c, C_MISC, "to_store", [&] { return launch_to_store(c->d_y, c->d_yh, cnt, v, c->stream); }));
            TRY(launch(c, C_MISC, "to_store", [&] { return launch_to_store(c->d_d, c->d_dh, cnt, v, c->stream); }));
        }
        c->store = v;
        CK(cudaStreamSynchronize(c->stream));
        return finish(c);
    }
    default: return fail(c, MC_EINVAL, "unknown option %d", option);
    }
}

mc_status mc_profile_read(mc_ctx* c, int32_t cap, const char** names, int64_t* counts, double* ms,
                          int32_t* n_out)
{
    if (!c) return MC_EINVAL;
    TRY(prof_collect(c));
    if (n_out) *n_out = kNumClasses;
    for (int i = 0; i < kNumClasses && i < cap; ++i) {
        if (names) names[i] = kClassNames[i];
        if (counts) counts[i] = c->prof_count[i];
        if (ms) ms[i] = c->prof_ms[i];
    }
    return MC_OK;
}

mc_status mc_profile_reset(mc_ctx* c)
{
    if (!c) return MC_EINVAL;
    TRY(prof_collect(c));
    for (int i = 0; i < kNumClasses; ++i) { c->prof_count[i] = 0; c->prof_ms[i] = 0; }
    return MC_OK;
}

// ---- checkpoint / resume -----------------------------------------------------
// Layout: header (8 x uint64) | x^K | x^{K+1} | z (n^2 float32 each) | y
// (N n_a n_b values of the current storage type: float32 or uint16).
namespace {
constexpr uint64_t kStateMagic = 0x3154535043474d4dULL;   // "MMGCPST1"
constexpr int kStateWords = 8;

size_t state_bytes(const mc_ctx* c)
{
    const size_t n2 = (size_t)c->n * c->n, ny = (size_t)c->N * c->na * c->nb;
    return kStateWords * sizeof(uint64_t) + 3 * n2 * sizeof(float) +
           ny * (c->store ? sizeof(unsigned short) : sizeof(float));
}
}  // namespace

mc_status mc_state_size(mc_ctx* c, uint64_t* bytes)
{
    if (!c || !bytes) return MC_EINVAL;
    *bytes = state_bytes(c);
    return MC_OK;
}

mc_status mc_save_state(mc_ctx* c, void* buf, uint64_t cap)
{
    if (!c) return MC_EINVAL;
    if (!buf) return fail(c, MC_EINVAL, "buf is NULL");
    if (ptr_kind(c, buf) != 0) return fail(c, MC_EINVAL, "buf must be host memory");
    const size_t need = state_bytes(c);
    if (cap < need) return fail(c, MC_EINVAL, "state needs %zu bytes, buffer has %llu", need, (unsigned long long)cap);
    const size_t n2 = (size_t)c->n * c->n, ny = (size_t)c->N * c->na * c->nb;
    uint64_t hdr[kStateWords] = {kStateMagic, (uint64_t)c->n, (uint64_t)c->na, (uint64_t)c->nb,
                                 (uint64_t)c->N, (uint64_t)c->store, (uint64_t)c->S, c->k_host};
    unsigned char* p = static_cast<unsigned char*>(buf);
    std::memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    CK(cudaMemcpyAsync(p, c->d_x[c->cur ^ 1], n2 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(p + n2 * sizeof(float), c->d_x[c->cur], n2 * sizeof(float), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaMemcpyAsync(p + 2 * n2 * sizeof(float), c->d_z, n2 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    unsigned char* py = p + 3 * n2 * sizeof(float);
    if (c->store)
        CK(cudaMemcpyAsync(py, c->d_yh, ny * sizeof(unsigned short), cudaMemcpyDeviceToHost, c->stream));
    else
        CK(cudaMemcpyAsync(py, c->d_y, ny * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return finish(c);
}

mc_status mc_load_state(mc_ctx* c, const void* buf, uint64_t size)
{
    if (!c) return MC_EINVAL;
    if (!buf) return fail(c, MC_EINVAL, "buf is NULL");
    if (ptr_kind(c, buf) != 0) return fail(c, MC_EINVAL, "buf must be host memory");
    if (size < kStateWords * sizeof(uint64_t)) return fail(c, MC_EINVAL, "state too short");
    uint64_t hdr[kStateWords];
    std::memcpy(hdr, buf, sizeof hdr);
    if (hdr[0] != kStateMagic) return fail(c, MC_EINVAL, "not a saved solver state");
    if (hdr[1] != (uint64_t)c->n || hdr[2] != (uint64_t)c->na || hdr[3] != (uint64_t)c->nb ||
        hdr[4] != (uint64_t)c->N)
        return fail(c, MC_EINVAL, "state is for geometry %llu x (%llu x %llu), %llu gates",
                    (unsigned long long)hdr[1], (unsigned long long)hdr[2], (unsigned long long)hdr[3],
                    (unsigned long long)hdr[4]);
    if (hdr[5] != (uint64_t)c->store || hdr[6] != (uint64_t)c->S)
        return fail(c, MC_EINVAL, "state was saved with storage %llu and %llu angle subsets (context: %d, %d)",
                    (unsigned long long)hdr[5], (unsigned long long)hdr[6], c->store, c->S);
    if (size < state_bytes(c)) return fail(c, MC_EINVAL, "state truncated");
    const size_t n2 = (size_t)c->n * c->n, ny = (size_t)c->N * c->na * c->nb;
    const unsigned char* p = static_cast<const unsigned char*>(buf) + kStateWords * sizeof(uint64_t);
    CK(cudaStreamSynchronize(c->stream));
    c->cur = 0;                                   // x^{K+1} in d_x[0], x^K in d_x[1]
    CK(cudaMemcpyAsync(c->d_x[1], p, n2 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_x[0], p + n2 * sizeof(float), n2 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_z, p + 2 * n2 * sizeof(float), n2 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    const unsigned char* py = p + 3 * n2 * sizeof(float);
    if (c->store)
        CK(cudaMemcpyAsync(c->d_yh, py, ny * sizeof(unsigned short), cudaMemcpyHostToDevice, c->stream));
    else
        CK(cudaMemcpyAsync(c->d_y, py, ny * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    const unsigned long long k = hdr[7];
    CK(cudaMemcpyAsync(c->d_k, &k, sizeof k, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->k_host = k;
    return finish(c);
}

mc_status mc_iteration(mc_ctx* c, uint64_t* out)
{
    if (!c || !out) return MC_EINVAL;
    *out = c->k_host;
    return MC_OK;
}

mc_status mc_sync(mc_ctx* c)
{
    if (!c) return MC_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    TRY(poll_err(c, true));
    TRY(check_err_word(c));
    return finish(c);
}

}  // extern "C"

// ============================================================================
// Batched SPDHG over many slices: one launch per stage of an iteration spans
// every slice in flight (per class of launch shape), replayed as CUDA graphs.
// ============================================================================
namespace {

// The launches of one batched iteration for the slices 0 .. A-1 of the
// batch's order (those still running): block maps per stage and class, and
// the captured graph of each parity of the iteration index.
// The forward blocks of the slices in flight that share one chunk size and
// ring (one compiled kernel): their block map range, the most group slots per
// warp among them and the largest ring.
struct FwdClass {
    size_t off = 0;
    int n = 0, rpt = 2, lc = 8, ns = 5, cl = 8;
    size_t smem = 0;
};

// The backprojection tiles of the slices in flight with one tile height.
struct BpClass {
    size_t off = 0;
    int n = 0, pj = 4;
};

struct BatchPhase {
    BatchBlock* d_map = nullptr;             // every map of the phase, one allocation
    int plan = 0;                            // forward work items: 0 each slice's own, 1 the batch's
    int n_warp = 0, n_wadj = 0;
    size_t off_warp = 0, off_wadj = 0;
    std::vector<FwdClass> fwd;               // one forward launch per class, classes concurrent
    std::vector<BpClass> bp;                 // one backprojection launch per tile height, likewise
    cudaGraphExec_t g[2][2] = {};            // [1 or kBatchGraphIters iterations][start parity]
};

constexpr int kBatchGraphIters = 16;         // batched iterations per replayed graph

}  // namespace

struct mc_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<mc_ctx*> ctx;                // caller's order
    std::vector<int> order;                  // slices by iterations per epoch, descending
    // per-slice argument tables in the order above ([t]: parity of the iteration index)
    WarpArgs* d_warp[2] = {nullptr, nullptr};
    FwdArgs* d_fwd[2][2] = {};               // [plan][t]; plan: the slice's own items, the batch's
    // the batch's forward work items per slice (order above): coarser than a
    // slice's own when its share of a merged launch is small, so that its
    // blocks stream its image once for many ray groups; used while enough
    // slices are in flight to fill the GPU (results do not depend on the cut)
    std::vector<int2*> d_bgroups;
    std::vector<RayItem*> d_bitems;
    std::vector<int> b_nitems, b_rpt;
    std::vector<char> b_owned;              // 0: the slice's own tables serve (no coarser cut)
    // each context's table generation, item count, chunk lines, rows per
    // thread and group slots at creation
    std::vector<std::array<long long, 5>> shape;
    BpArgs* d_bp[2] = {nullptr, nullptr};
    WarpAdjArgs* d_wadj[2] = {nullptr, nullptr};
    BatchDraw* d_draw = nullptr;
    int* d_state = nullptr;                  // per slice [2][2]: {iteration in epoch, epoch parity}
    int* d_bgates = nullptr;                 // per slice two epochs of gates, stride gmax
    int gmax = 1;
    std::vector<unsigned long long> k_end;   // each slice's counter after a run (host copy source)
    // with one slice in flight (order[0]) the one-slice kernels run on copies
    // of its table rows, passed by value (baked into that phase's graphs)
    WarpArgs h_warp[2] = {};
    FwdArgs h_fwd[2][2] = {};
    BpArgs h_bp[2] = {};
    WarpAdjArgs h_wadj[2] = {};
    std::vector<BatchPhase> phase;           // [A - 1] for A slices in flight, built on demand
    std::vector<cudaEvent_t> ev;             // one per slice (hand-off between streams) + 1
    // forward classes after the first run on side streams: a fork before and a
    // join after (graph branches once captured)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
};

namespace {

mc_status bfail(mc_batch* b, mc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return st;
}

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bfail(b, MC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

void batch_free(mc_batch* b)
{
    for (auto& ph : b->phase) {
        for (auto& row : ph.g)
            for (auto& g : row)
                if (g) cudaGraphExecDestroy(g);
        if (ph.d_map) cudaFree(ph.d_map);
    }
    b->phase.clear();
    for (void* p : {(void*)b->d_warp[0], (void*)b->d_warp[1], (void*)b->d_fwd[0][0], (void*)b->d_fwd[0][1],
                    (void*)b->d_fwd[1][0], (void*)b->d_fwd[1][1], (void*)b->d_bp[0], (void*)b->d_bp[1],
                    (void*)b->d_wadj[0], (void*)b->d_wadj[1], (void*)b->d_draw, (void*)b->d_state,
                    (void*)b->d_bgates})
        if (p) cudaFree(p);
    for (size_t q = 0; q < b->d_bgroups.size(); ++q)
        if (q < b->b_owned.size() && b->b_owned[q]) {
            if (b->d_bgroups[q]) cudaFree(b->d_bgroups[q]);
            if (b->d_bitems[q]) cudaFree(b->d_bitems[q]);
        }
    b->b_owned.clear();
    b->d_bgroups.clear();
    b->d_bitems.clear();
    for (auto e : b->ev) cudaEventDestroy(e);
    b->ev.clear();
    for (auto e : b->join_ev) cudaEventDestroy(e);
    b->join_ev.clear();
    for (auto q : b->side) cudaStreamDestroy(q);
    b->side.clear();
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    b->fork_ev = nullptr;
}

template <class T>
mc_status balloc(mc_batch* b, T** p, size_t count)
{
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, MC_ENOMEM, "cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    *p = static_cast<T*>(q);
    return MC_OK;
}

// Fill the per-slice argument tables from the contexts' current state (step
// sizes, storage, sampling, parity of x): exactly the arguments the
// one-slice epoch of enqueue_spdhg_epoch gives its kernels, with the drawn
// gate read through the slice's epoch position.
mc_status batch_tables(mc_batch* b, const mc_sampling* sampling)
{
    const int B = (int)b->order.size();
    std::vector<WarpArgs> w[2];
    std::vector<WarpAdjArgs> wa[2];
    std::vector<FwdArgs> f[2][2];
    std::vector<BpArgs> bp[2];
    std::vector<BatchDraw> dr(B);
    for (int t = 0; t < 2; ++t) {
        w[t].resize(B); wa[t].resize(B); bp[t].resize(B);
        f[0][t].resize(B); f[1][t].resize(B);
    }
    for (int q = 0; q < B; ++q) {
        mc_ctx* c = b->ctx[b->order[q]];
        const bool nonuni = !c->p_steps.empty();
        int* gates = b->d_bgates + (size_t)q * 2 * b->gmax;
        int* state = b->d_state + 4 * (size_t)q;
        for (int t = 0; t < 2; ++t) {
            // the drawn gate of an iteration of parity t: gates[epar * gmax + pos], state[t] = {pos, epar}
            const GateSel sel{gates, -1, 1, state + 2 * t, b->gmax};
            WarpArgs& a = w[t][q];
            a = WarpArgs{};
            a.x = c->d_x[c->cur ^ t]; a.n = c->n;
            a.rigid = c->d_rigid; a.field = c->d_field; a.identity = 0;
            a.sel = sel; a.n_slots = 1;
            a.lrow = c->d_lrow; a.lcol = c->d_lcol; a.layout_stride = c->layout_stride; a.P = c->P;
            a.guard = c->guard;
            WarpAdjArgs& u = wa[t][q];
            u = wadj_args(c, sel, 1, c->d_b);
            u.z = c->d_z; u.x_in = c->d_x[c->cur ^ t]; u.x_out = c->d_x[c->cur ^ t ^ 1];
            u.coef = (float)(c->sS.theta * c->N);
            u.coef_tab = nonuni ? c->d_coef : nullptr;
            u.tau = (float)c->sS.tau;
            u.prox_scale = (float)(1.0 / (1.0 + 2.0 * c->sS.tau * c->alpha));
            FwdArgs& fa = f[0][t][q];
            fa = FwdArgs{};
            fa.lrow = c->d_lrow; fa.lcol = c->d_lcol; fa.layout_stride = c->layout_stride; fa.P = c->P;
            fa.guard = c->guard;
            fa.ang = c->d_fang; fa.groups = c->d_groups; fa.items = c->d_items; fa.n_items = c->n_items;
            fa.ipb = c->ipb; fa.rpt = c->rpt; fa.lc = c->lc; fa.n = c->n; fa.na = c->na; fa.nb = c->nb;
            fa.stages = forward_ring(c->lc, c->P);
            fa.cl = forward_part_lines(c->lc, c->guard);
            fa.sel = sel; fa.n_slots = 1; fa.wait_limit = 1u << 24;
            fa.dy = c->d_dy; fa.dy_stride = c->dy_stride; fa.Pb = c->Pb; fa.Gb = c->Gb; fa.err = c->d_err;
            fa.mode = 1; fa.d = c->d_d; fa.y = c->d_y;
            fa.sigma = (float)c->sS.sigma;
            fa.inv_den = (float)(1.0 / (1.0 + c->sS.sigma * c->N / 2.0));
            fa.pf_rowptr = c->d_rowptr; fa.pf_ent = c->d_ent; fa.pf_ent_off = c->d_ent_off;
            fa.store = c->store; fa.dh = c->d_dh; fa.yh = c->d_yh;
            FwdArgs& f1 = f[1][t][q];
            f1 = fa;
            f1.groups = b->d_bgroups[q]; f1.items = b->d_bitems[q]; f1.n_items = b->b_nitems[q];
            f1.ipb = 1; f1.rpt = b->b_rpt[q];
            BpArgs& g = bp[t][q];
            g = BpArgs{};
            g.sel = sel;
            g.dy = c->d_dy; g.dy_stride = c->dy_stride; g.Pb = c->Pb; g.Gb = c->Gb;
            g.ang = c->d_bang; g.n = c->n; g.na = c->na; g.nb = c->nb; g.n_slots = 1;
            g.pj = c->pj; g.out = c->d_b; g.err = c->d_err; g.wl = backproject_window(c->pj);
            if (g.wl > g.Pb)
                return bfail(b, MC_EINVAL, "slice %d: backprojection window wider than its dual layout", b->order[q]);
        }
        const mc_sampling& sm = sampling[b->order[q]];
        dr[q] = BatchDraw{sm.seed, sm.stream, c->N, c->d_k, nonuni ? c->d_thr : nullptr, gates, state, b->gmax};
    }
    for (int t = 0; t < 2; ++t) {
        BCK(cudaMemcpy(b->d_warp[t], w[t].data(), B * sizeof(WarpArgs), cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(b->d_wadj[t], wa[t].data(), B * sizeof(WarpAdjArgs), cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(b->d_bp[t], bp[t].data(), B * sizeof(BpArgs), cudaMemcpyHostToDevice));
        for (int k = 0; k < 2; ++k)
            BCK(cudaMemcpy(b->d_fwd[k][t], f[k][t].data(), B * sizeof(FwdArgs), cudaMemcpyHostToDevice));
    }
    BCK(cudaMemcpy(b->d_draw, dr.data(), B * sizeof(BatchDraw), cudaMemcpyHostToDevice));
    // the one-slice phase's arguments by value: its graphs go when they change
    for (int t = 0; t < 2; ++t) {
        wa[t][0].draw = b->d_draw;
        wa[t][0].draw_t = t;
    }
    const WarpArgs nw[2] = {w[0][0], w[1][0]};
    const BpArgs nb[2] = {bp[0][0], bp[1][0]};
    const WarpAdjArgs nwa[2] = {wa[0][0], wa[1][0]};
    const FwdArgs nf[2][2] = {{f[0][0][0], f[0][1][0]}, {f[1][0][0], f[1][1][0]}};
    const bool same = !memcmp(b->h_warp, nw, sizeof nw) && !memcmp(b->h_bp, nb, sizeof nb) &&
                      !memcmp(b->h_wadj, nwa, sizeof nwa) && !memcmp(b->h_fwd, nf, sizeof nf);
    if (!same && !b->phase.empty())
        for (auto& row : b->phase[0].g)
            for (auto& g : row)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    memcpy(b->h_warp, nw, sizeof nw);
    memcpy(b->h_bp, nb, sizeof nb);
    memcpy(b->h_wadj, nwa, sizeof nwa);
    memcpy(b->h_fwd, nf, sizeof nf);
    return MC_OK;
}

// Block maps of the iteration with slices order[0 .. A-1] in flight.  Each
// stage is one launch listing every such slice's blocks (for the forward the
// batch's coarser items while they fill the GPU, else the slice's own), slices
// with more work per block first so that the block scheduler ends the launch
// with the small ones; each block runs with its slice's launch shape (lines
// per chunk, rows per thread).
mc_status batch_phase(mc_batch* b, int A)
{
    BatchPhase& ph = b->phase[A - 1];
    if (ph.d_map) return MC_OK;
    std::vector<int> q(A);
    for (int i = 0; i < A; ++i) q[i] = i;
    auto C = [&](int i) { return b->ctx[b->order[i]]; };
    std::vector<BatchBlock> all;
    auto add = [&](std::vector<int> qs, auto blocks_of, auto work_of) {
        std::stable_sort(qs.begin(), qs.end(), [&](int x, int y) { return work_of(x) > work_of(y); });
        const size_t off = all.size();
        for (int i : qs) {
            const int nbk = blocks_of(i);
            for (int k = 0; k < nbk; ++k) all.push_back(BatchBlock{i, k, nbk, 0});
        }
        return std::make_pair(off, (int)(all.size() - off));
    };
    // warp: tiles of 32 x 30 pixels, equal work
    {
        auto r = add(q, [&](int i) { return warp_layout_tiles(C(i)->n); }, [&](int) { return 0.0; });
        ph.off_warp = r.first; ph.n_warp = r.second;
    }
    // forward: the batch's coarser work items while they still give every SM
    // a few blocks, else each slice's own; one class (and launch) per chunk
    // size and ring; a block's work ~ samples / blocks
    {
        long long coarse = 0;
        for (int i : q) coarse += b->b_nitems[i];
        ph.plan = coarse >= 4LL * b->ctx[0]->sms ? 1 : 0;
    }
    auto f_blocks = [&](int i) {
        return ph.plan ? b->b_nitems[i] : (C(i)->n_items + C(i)->ipb - 1) / C(i)->ipb;
    };
    auto f_rpt = [&](int i) { return ph.plan ? b->b_rpt[i] : C(i)->rpt; };
    {
        std::vector<std::array<int, 3>> keys;           // (lc, ring stages, part lines), in order
        std::vector<std::vector<int>> members;
        for (int i : q) {
            const std::array<int, 3> k{C(i)->lc, forward_ring(C(i)->lc, C(i)->P),
                                       forward_part_lines(C(i)->lc, C(i)->guard)};
            size_t j = 0;
            while (j < keys.size() && keys[j] != k) ++j;
            if (j == keys.size()) { keys.push_back(k); members.emplace_back(); }
            members[j].push_back(i);
        }
        ph.fwd.clear();
        for (size_t j = 0; j < keys.size(); ++j) {
            FwdClass fc;
            fc.lc = keys[j][0];
            fc.ns = keys[j][1];
            fc.cl = keys[j][2];
            for (int i : members[j]) {
                fc.rpt = std::max(fc.rpt, f_rpt(i));
                fc.smem = std::max(fc.smem, forward_smem_bytes(C(i)->lc, C(i)->P));
            }
            auto r = add(members[j], f_blocks, [&](int i) {
                const mc_ctx* c = C(i);
                return (double)c->na * c->n * c->n / f_blocks(i);
            });
            fc.off = r.first;
            fc.n = r.second;
            ph.fwd.push_back(fc);
        }
    }
    // backprojection: one class per tile height; a tile's work ~ angles x rows
    {
        std::vector<int> heights;
        for (int i : q)
            if (std::find(heights.begin(), heights.end(), C(i)->pj) == heights.end()) heights.push_back(C(i)->pj);
        ph.bp.clear();
        for (int pj : heights) {
            std::vector<int> members;
            for (int i : q)
                if (C(i)->pj == pj) members.push_back(i);
            auto r = add(members, [&](int i) { return backproject_tiles(C(i)->n, C(i)->pj); },
                         [&](int i) { return (double)C(i)->na * C(i)->pj; });
            BpClass bc;
            bc.off = r.first;
            bc.n = r.second;
            bc.pj = pj;
            ph.bp.push_back(bc);
        }
    }
    {
        // side streams and events for the classes after the first of either stage
        const size_t classes = std::max(ph.fwd.size(), ph.bp.size());
        while (b->side.size() + 1 < classes) {
            cudaStream_t q2 = nullptr;
            cudaEvent_t e2 = nullptr;
            BCK(cudaStreamCreateWithFlags(&q2, cudaStreamNonBlocking));
            b->side.push_back(q2);
            BCK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
            b->join_ev.push_back(e2);
        }
        if (classes > 1 && !b->fork_ev) BCK(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
    }
    // transpose warp and update: 256 pixels per block
    {
        auto r = add(q, [&](int i) { return warp_adjoint_blocks(C(i)->n); }, [&](int) { return 0.0; });
        ph.off_wadj = r.first; ph.n_wadj = r.second;
    }
    if (balloc(b, &ph.d_map, all.size()) != MC_OK) return MC_ENOMEM;
    BCK(cudaMemcpy(ph.d_map, all.data(), all.size() * sizeof(BatchBlock), cudaMemcpyHostToDevice));
    return MC_OK;
}

// Enqueue `iters` batched iterations, the first of parity t, for the slices
// of phase A on the batch's stream: four launches each (the gate sequence
// advances inside the last one).
mc_status batch_enqueue(mc_batch* b, int A, int t, int iters)
{
    BatchPhase& ph = b->phase[A - 1];
    cudaStream_t s = b->stream;
    for (int i = 0; i < iters; ++i, t ^= 1) {
        if (A == 1) {
            // one slice in flight: the one-slice kernels, arguments by value
            BCK(launch_warp_layouts(b->h_warp[t], s));
            BCK(launch_forward(b->h_fwd[ph.plan][t], s));
            BCK(launch_backproject(b->h_bp[t], s));
            BCK(launch_warp_adjoint_update(b->h_wadj[t], s));
            continue;
        }
        BCK(launch_warp_layouts_batch(b->d_warp[t], ph.d_map + ph.off_warp, ph.n_warp, s));
        // the forward: one launch per class, the classes after the first on
        // side streams between a fork and a join, so that they run together
        const FwdArgs* fa = b->d_fwd[ph.plan][t];
        if (ph.fwd.size() > 1) BCK(cudaEventRecord(b->fork_ev, s));
        for (size_t k = 1; k < ph.fwd.size(); ++k) {
            const FwdClass& fc = ph.fwd[k];
            cudaStream_t q2 = b->side[k - 1];
            BCK(cudaStreamWaitEvent(q2, b->fork_ev, 0));
            BCK(launch_forward_batch(fa, ph.d_map + fc.off, fc.n, fc.rpt, fc.smem, fc.lc, fc.ns, fc.cl, q2));
            BCK(cudaEventRecord(b->join_ev[k - 1], q2));
        }
        const FwdClass& f0 = ph.fwd[0];
        BCK(launch_forward_batch(fa, ph.d_map + f0.off, f0.n, f0.rpt, f0.smem, f0.lc, f0.ns, f0.cl, s));
        for (size_t k = 1; k < ph.fwd.size(); ++k) BCK(cudaStreamWaitEvent(s, b->join_ev[k - 1], 0));
        // the backprojection: one launch per tile height, the same way
        if (ph.bp.size() > 1) BCK(cudaEventRecord(b->fork_ev, s));
        for (size_t k = 1; k < ph.bp.size(); ++k) {
            const BpClass& bc = ph.bp[k];
            cudaStream_t q2 = b->side[k - 1];
            BCK(cudaStreamWaitEvent(q2, b->fork_ev, 0));
            BCK(launch_backproject_batch(b->d_bp[t], ph.d_map + bc.off, bc.n, bc.pj, q2));
            BCK(cudaEventRecord(b->join_ev[k - 1], q2));
        }
        BCK(launch_backproject_batch(b->d_bp[t], ph.d_map + ph.bp[0].off, ph.bp[0].n, ph.bp[0].pj, s));
        for (size_t k = 1; k < ph.bp.size(); ++k) BCK(cudaStreamWaitEvent(s, b->join_ev[k - 1], 0));
        BCK(launch_warp_adjoint_update_batch(b->d_wadj[t], ph.d_map + ph.off_wadj, ph.n_wadj, b->d_draw, t, s));
    }
    return MC_OK;
}

}  // namespace

extern "C" {

mc_status mc_batch_create(mc_ctx* const* ctxs, int32_t count, void* cuda_stream, mc_batch** out)
{
    if (!out || !ctxs || count < 1) return MC_EINVAL;
    *out = nullptr;
    mc_batch* b = new mc_batch();
    for (int i = 0; i < count; ++i) {
        mc_ctx* c = ctxs[i];
        if (!c) { delete b; return MC_EINVAL; }
        if (i == 0) b->dev = c->dev;
        if (c->dev != b->dev) { delete b; return fail(c, MC_EINVAL, "batch contexts must share one device"); }
        if (c->S != 1) { delete b; return fail(c, MC_EINVAL, "batched runs sample gates only (subsets = 1)"); }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) { delete b; return fail(c, MC_EINVAL, "a context appears twice in the batch"); }
        b->ctx.push_back(c);
    }
    mc_status st = MC_OK;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        cudaGetLastError();
        delete b;
        return MC_ECUDA;
    }
    // slices by iterations per epoch (N), then by size: the slices in flight
    // are always a prefix of this order
    for (int i = 0; i < count; ++i) b->order.push_back(i);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        const mc_ctx *p = b->ctx[x], *q = b->ctx[y];
        if (p->N != q->N) return p->N > q->N;
        return (double)p->na * p->n * p->n > (double)q->na * q->n * q->n;
    });
    for (int t = 0; t < 2 && st == MC_OK; ++t) {
        st = balloc(b, &b->d_warp[t], count);
        if (st == MC_OK) st = balloc(b, &b->d_wadj[t], count);
        if (st == MC_OK) st = balloc(b, &b->d_bp[t], count);
        if (st == MC_OK) st = balloc(b, &b->d_fwd[0][t], count);
        if (st == MC_OK) st = balloc(b, &b->d_fwd[1][t], count);
    }
    for (auto* c : b->ctx) b->gmax = std::max(b->gmax, c->N);
    if (st == MC_OK) st = balloc(b, &b->d_state, 4 * (size_t)count);
    if (st == MC_OK) st = balloc(b, &b->d_bgates, 2 * (size_t)count * b->gmax);
    // the batch's forward work items: about 4 blocks per SM over the whole
    // batch, each slice's share by its samples per projection, at least as
    // many items as its groups need (at most forward_warps warps x 8 slots
    // each) and at most as many as its own plan has
    if (st == MC_OK) {
        const int sms = b->ctx[0]->sms;
        double W = 0;
        for (auto* c : b->ctx) W += (double)c->na * c->n * c->n;
        b->d_bgroups.assign(count, nullptr);
        b->d_bitems.assign(count, nullptr);
        b->b_nitems.assign(count, 0);
        b->b_rpt.assign(count, 2);
        b->b_owned.assign(count, 0);
        for (int q = 0; q < count; ++q) {
            const mc_ctx* c = b->ctx[b->order[q]];
            b->shape.push_back({(long long)c->tables_gen, c->n_items, c->lc, c->pj, c->rpt});
        }
        for (int q = 0; q < count && st == MC_OK; ++q) {
            mc_ctx* c = b->ctx[b->order[q]];
            const double share = (double)c->na * c->n * c->n / W;
            const int own = (c->n_items + c->ipb - 1) / c->ipb;
            const int target = std::max(1, std::min(own, (int)std::lround(4.0 * sms * share)));
            if (c->ipb == 1 && 2 * target > own) {
                // no worthwhile coarsening: the slice's own items serve
                b->d_bgroups[q] = c->d_groups;
                b->d_bitems[q] = c->d_items;
                b->b_nitems[q] = c->n_items;
                b->b_rpt[q] = c->rpt;
                continue;
            }
            b->b_owned[q] = 1;
            GroupTable gt;
            build_groups(c, 1, c->lc, gt);
            std::vector<RayItem> items;
            std::vector<int> off;
            int ipb = 1, rpt = 2;
            plan_forward(c, c->lc, target, 1, kPlanRounds, gt, items, off, ipb, rpt);
            // one item per block: ipb items of the cut are ipb blocks
            st = balloc(b, &b->d_bgroups[q], gt.groups.size());
            if (st == MC_OK) st = balloc(b, &b->d_bitems[q], items.size());
            if (st == MC_OK &&
                (cudaMemcpy(b->d_bgroups[q], gt.groups.data(), gt.groups.size() * sizeof(int2),
                            cudaMemcpyHostToDevice) != cudaSuccess ||
                 cudaMemcpy(b->d_bitems[q], items.data(), items.size() * sizeof(RayItem),
                            cudaMemcpyHostToDevice) != cudaSuccess)) {
                cudaGetLastError();
                st = MC_ECUDA;
            }
            b->b_nitems[q] = (int)items.size();
            b->b_rpt[q] = rpt;
        }
    }
    if (st == MC_OK) st = balloc(b, &b->d_draw, count);
    b->phase.resize(count);
    for (int i = 0; i <= count && st == MC_OK; ++i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            st = MC_ECUDA;
        } else {
            b->ev.push_back(e);
        }
    }
    if (st != MC_OK) {
        batch_free(b);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return st;
    }
    *out = b;
    return MC_OK;
}

const char* mc_batch_last_error(const mc_batch* b) { return b ? b->err.c_str() : ""; }

void mc_batch_destroy(mc_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

mc_status mc_batch_run(mc_batch* b, int32_t epochs, const mc_sampling* sampling, int32_t* failed)
{
    if (failed) *failed = -1;
    if (!b) return MC_EINVAL;
    if (!sampling) return bfail(b, MC_EINVAL, "sampling is NULL");
    if (epochs < 0) return bfail(b, MC_EINVAL, "epochs must be >= 0");
    const int B = (int)b->ctx.size();
    for (int i = 0; i < B; ++i) {
        mc_ctx* c = b->ctx[i];
        mc_status st = MC_OK;
        if (!c->have_data || !c->steps_ok)
            st = fail(c, MC_ESTATE, "runs need mc_set_data and mc_norms/mc_set_norms first");
        else if (c->S != 1)
            st = fail(c, MC_EINVAL, "batched runs sample gates only (subsets = 1)");
        if (st == MC_OK) st = apply_sampling(c, &sampling[i]);
        if (st != MC_OK) {
            if (failed) *failed = i;
            return bfail(b, st, "slice %d: %s", i, c->err.c_str());
        }
    }
    for (int q = 0; q < B; ++q) {
        const mc_ctx* c = b->ctx[b->order[q]];
        const std::array<long long, 5> now{(long long)c->tables_gen, c->n_items, c->lc, c->pj, c->rpt};
        if (now != b->shape[q]) {
            if (failed) *failed = b->order[q];
            return bfail(b, MC_ESTATE, "slice %d: its launch shapes changed after mc_batch_create "
                                      "(mc_autotune or a shape option); create the batch again",
                         b->order[q]);
        }
    }
    if (epochs == 0) return MC_OK;
    // the batch's stream starts after every slice's own pending work
    for (int i = 0; i < B; ++i) {
        BCK(cudaEventRecord(b->ev[i], b->ctx[i]->stream));
        BCK(cudaStreamWaitEvent(b->stream, b->ev[i], 0));
    }
    // the tables are read by the graphs at run time: no graph is recaptured
    // for new step sizes, seeds or sampling
    BCK(cudaStreamSynchronize(b->stream));
    TRY(batch_tables(b, sampling));
    // every slice starts an epoch: state[0] = {0, 0} and its first epoch's
    // gates drawn into the first half from its counter, as the one-slice
    // epoch does
    std::vector<int> st0(4 * (size_t)B, 0);
    std::vector<long long> iters(B);
    BCK(cudaMemcpyAsync(b->d_state, st0.data(), st0.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    for (int q = 0; q < B; ++q) {
        mc_ctx* c = b->ctx[b->order[q]];
        iters[q] = (long long)epochs * c->N;
        const mc_sampling& sm = sampling[b->order[q]];
        BCK(launch_draw_gates(sm.seed, sm.stream, c->d_k, 0, c->N, c->N, c->p_steps.empty() ? nullptr : c->d_thr,
                              b->d_bgates + (size_t)q * 2 * b->gmax, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));           // the state copied from the host vector
    auto graph_for = [&](BatchPhase& ph, int A, int size_i, int t) -> mc_status {
        cudaGraphExec_t& ge = ph.g[size_i][t];
        if (ge) return MC_OK;
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const mc_status st = batch_enqueue(b, A, t, size_i ? kBatchGraphIters : 1);
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st != MC_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return bfail(b, MC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return bfail(b, MC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e2));
        return MC_OK;
    };
    long long done = 0;
    int A = B;
    while (A > 0) {
        // the iterations in which exactly the first A slices are in flight,
        // kBatchGraphIters per graph launch (an even count: the parity repeats)
        const long long end = iters[A - 1];
        if (end > done) {
            TRY(batch_phase(b, A));
            BatchPhase& ph = b->phase[A - 1];
            long long it = done;
            while (it < end) {
                const int t = (int)(it & 1);
                const int size_i = (end - it >= kBatchGraphIters) ? 1 : 0;
                TRY(graph_for(ph, A, size_i, t));
                BCK(cudaGraphLaunch(ph.g[size_i][t], b->stream));
                it += size_i ? kBatchGraphIters : 1;
            }
            done = end;
        }
        --A;
    }
    // each slice's counter as its own runs leave it (the last iteration of a
    // slice drew an epoch it does not run)
    b->k_end.resize(B);
    for (int q = 0; q < B; ++q) {
        mc_ctx* c = b->ctx[b->order[q]];
        b->k_end[q] = (unsigned long long)(c->k_host + (uint64_t)iters[q]);
        BCK(cudaMemcpyAsync(c->d_k, &b->k_end[q], sizeof(unsigned long long), cudaMemcpyHostToDevice, b->stream));
    }
    // every slice's own stream continues after the batch
    BCK(cudaEventRecord(b->ev[B], b->stream));
    for (int i = 0; i < B; ++i) BCK(cudaStreamWaitEvent(b->ctx[i]->stream, b->ev[B], 0));
    BCK(cudaStreamSynchronize(b->stream));
    for (int q = 0; q < B; ++q) {
        mc_ctx* c = b->ctx[b->order[q]];
        c->k_host += (uint64_t)iters[q];
        c->cur ^= (int)(iters[q] & 1);
    }
    for (int i = 0; i < B; ++i) {
        mc_ctx* c = b->ctx[i];
        mc_status st = check_err_word(c);
        if (st == MC_OK) st = finish(c);
        if (st != MC_OK) {
            if (failed) *failed = i;
            return bfail(b, st, "slice %d: %s", i, c->err.c_str());
        }
    }
    return MC_OK;
}

}  // extern "C"
