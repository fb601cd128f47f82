// mc_forward_static: the forward operator A D of one motion state for callers
// that cannot allocate device memory (for example code running inside an
// allocator hook, a memory-capped plugin, or a host that has already handed
// every byte of the GPU to its own pool).  All scratch -- angle and ray-group
// tables, the two line layouts of the warped image, the error word -- lives
// in one fixed, file-scope device array, so the call performs no cudaMalloc,
// cudaFree or other allocation.  The work itself is the same warp and Joseph
// projection kernels that mc_forward uses.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "mc.h"
#include "mc_kernels.h"

using namespace mcg;

namespace {

constexpr size_t kStaticScratchBytes = size_t(24) << 20;   // 24 MiB per device
constexpr int kMaxDevices = 64;
constexpr double kPiD = 3.14159265358979323846;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

void set_msg(char* err, int cap, const char* fmt, ...)
{
    if (!err || cap <= 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, (size_t)cap, fmt, ap);
    va_end(ap);
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Scratch layout (byte offsets into g_scratch), every region 256-aligned.
struct Layout {
    size_t err, rigid, ang, groups, items, lrow, lcol, total;
};

Layout layout_for(int n, int na, int nb, int P, int n_items)
{
    const int gpa = (nb + 31) / 32;
    Layout L{};
    size_t o = 0;
    L.err = o;    o += align256(sizeof(int));
    L.rigid = o;  o += align256(sizeof(RigidGate));
    L.ang = o;    o += align256((size_t)na * sizeof(FwdAngle));
    L.groups = o; o += align256((size_t)na * gpa * sizeof(int2));
    L.items = o;  o += align256((size_t)n_items * sizeof(RayItem));
    L.lrow = o;   o += align256((size_t)layout_lines(n) * P * sizeof(float2));
    L.lcol = o;   o += align256((size_t)layout_lines(n) * P * sizeof(float2));
    L.total = o;
    return L;
}

__device__ __forceinline__ void split_d(double v, float& hi, float& lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Tables of one call, built on the device from the geometry (float64), so that
// no host buffer has to be staged: the Joseph table of every angle, the ray
// groups in angle order (rows-driven angles first), items of at most gpi
// consecutive groups per axis class, and the rigid map.
__global__ void k_static_tables(int n, int na, int nb, int lc, int gpi, int items0,
                                int rigid_on, double phi, double tx, double ty,
                                FwdAngle* ang, int2* groups, RayItem* items, RigidGate* rg)
{
    const int gpa = (nb + 31) / 32;
    const int kx0 = (na + 3) / 4;                  // first columns-driven angle
    const int kx1 = (3 * na) / 4;                  // last columns-driven angle
    const int ny = kx0 + (na - 1 - kx1);           // rows-driven angles
    const int n_groups = na * gpa;
    const int items1 = (na - ny) * gpa > 0 ? ((na - ny) * gpa + gpi - 1) / gpi : 0;
    const int stride = gridDim.x * blockDim.x;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < na + n_groups + items0 + items1 + 1; t += stride) {
        if (t < na) {
            const int k = t;
            const double p = (double)k * kPiD / (double)na;
            const double cs = cos(p), sn = sin(p);
            const bool xd = (na <= 4 * k) && (4 * k <= 3 * na);
            const double inv = xd ? 1.0 / sn : 1.0 / cs;
            const double tt = xd ? cs / sn : sn / cs;
            FwdAngle f;
            split_d(inv, f.inv_hi, f.inv_lo);
            split_d(tt, f.t_hi, f.t_lo);
            const double step = (double)lc * tt;
            const double si = floor(step);
            f.step_int = (int)si;
            f.step_frac = (float)(step - si);
            if (f.step_frac >= 1.0f) { f.step_frac = 0.0f; f.step_int += 1; }
            f.delta = (float)fabs(inv);
            f.dir = xd ? 1 : 0;
            ang[k] = f;
        } else if (t < na + n_groups) {
            const int gi = t - na;
            const int o = gi / gpa, g = gi - o * gpa;
            int k;
            if (o < ny) k = (o < kx0) ? o : kx1 + 1 + (o - kx0);
            else k = kx0 + (o - ny);
            groups[gi] = make_int2(k, g * 32);
        } else if (t < na + n_groups + items0 + items1) {
            const int i = t - na - n_groups;
            const int cls = i < items0 ? 0 : 1;
            const int b0 = cls == 0 ? 0 : ny * gpa, b1 = cls == 0 ? ny * gpa : n_groups;
            const int j = cls == 0 ? i : i - items0;
            items[i] = RayItem{b0 + j * gpi, min(b1, b0 + (j + 1) * gpi), cls, 0};
        } else {
            RigidGate g;
            const double h = 0.5 * (n - 1);
            const double c = rigid_on ? cos(phi) : 1.0, s = rigid_on ? sin(phi) : 0.0;
            split_d(c, g.cos_hi, g.cos_lo);
            split_d(s, g.sin_hi, g.sin_lo);
            split_d((rigid_on ? tx : 0.0) + h, g.offx_hi, g.offx_lo);
            split_d((rigid_on ? ty : 0.0) + h, g.offy_hi, g.offy_lo);
            *rg = g;
        }
    }
}

// Per-device set-up under the lock: the device address of the scratch array
// (the host-side symbol is only a stand-in and must never reach a kernel) and,
// once per device, the forward kernels' shared-memory attribute.  The address
// is looked up again on every call made outside stream capture (a cheap
// query that allocates nothing), so a device or primary-context reset by the
// host application cannot leave a stale pointer behind; inside a capture the
// address of the last call made outside one is used.
mc_status device_setup(int dev, bool capturing, void** ptr, int* sms, char* err, int cap)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        set_msg(err, cap, "device %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
        return MC_EDEVICE;
    }
    if (capturing && !g_ptr[dev]) {
        set_msg(err, cap, "the first call on a device must come before any stream capture");
        return MC_ESTATE;
    }
    if (!capturing) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_msg(err, cap, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return MC_ECUDA;
        }
        if (p != g_ptr[dev]) g_sms[dev] = 0;     // new context: attributes again
        g_ptr[dev] = p;
    }
    if (!g_sms[dev]) {
        cudaError_t e;
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        e = forward_prepare(optin - forward_static_smem());
        if (e != cudaSuccess) {
            set_msg(err, cap, "cudaFuncSetAttribute failed: %s", cudaGetErrorString(e));
            return MC_ECUDA;
        }
        int s = 0;
        cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = s > 0 ? s : 1;
    }
    *ptr = g_ptr[dev];
    *sms = g_sms[dev];
    return MC_OK;
}

// MC_STATIC_TEST_STALL=1 in the environment (read at every call) makes the
// projection's waits run out, so that tests can check that the failure is
// reported by mc_forward_static_status.
bool stall_requested()
{
    const char* v = std::getenv("MC_STATIC_TEST_STALL");
    return v && v[0] == '1';
}

bool on_device(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" mc_status mc_forward_static(const mc_geometry* geom, const double* rigid, const float* x,
                                       float* out, void* cuda_stream, char* err, int32_t err_cap)
{
    if (err && err_cap > 0) err[0] = '\0';
    if (!geom || !x || !out) {
        set_msg(err, err_cap, "geometry, x and out are required");
        return MC_EINVAL;
    }
    const int n = geom->n, na = geom->n_angles, nb = geom->n_bins;
    if (n < 2 || n > 2048 || na < 1 || na > 8192 || nb < 1 || nb > 8192) {
        set_msg(err, err_cap, "geometry n=%d n_angles=%d n_bins=%d outside [2,2048] x [1,8192] x [1,8192]",
                n, na, nb);
        return MC_EINVAL;
    }
    if (rigid && !(std::isfinite(rigid[0]) && std::isfinite(rigid[1]) && std::isfinite(rigid[2]))) {
        set_msg(err, err_cap, "rigid motion is not finite");
        return MC_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_msg(err, err_cap, "no CUDA device");
        return MC_EDEVICE;
    }
    if (!on_device(x, dev) || !on_device(out, dev)) {
        set_msg(err, err_cap, "x and out must be device memory of the current device");
        return MC_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap_st) != cudaSuccess) {
        cudaGetLastError();
        set_msg(err, err_cap, "invalid stream");
        return MC_EINVAL;
    }
    void* base = nullptr;
    int sms = 1;
    mc_status st = device_setup(dev, cap_st != cudaStreamCaptureStatusNone, &base, &sms, err, err_cap);
    if (st != MC_OK) return st;

    // sizes: same line pitch and chunking as the context path; items of at
    // most gpi groups, gpi sized for one block per SM
    const int P = layout_pitch(n, kGuardNarrow);
    const int lc = std::min(8, forward_default_lines(n, P, kGuardNarrow));   // chunks sampled whole
    const int gpa = (nb + 31) / 32;
    const int kx0 = (na + 3) / 4, kx1 = (3 * na) / 4;
    const int ny = kx0 + (na - 1 - kx1);
    const long long n_groups = (long long)na * gpa;
    int rpt = 2;
    long long gpi = (n_groups + sms - 1) / sms;
    const int warps = forward_warps(lc, lc);   // chunks sampled whole
    while (rpt < 8 && forward_groups_per_block(rpt, warps) < gpi) rpt <<= 1;
    gpi = std::min<long long>(gpi, forward_groups_per_block(rpt, warps));
    const int items0 = (int)(((long long)ny * gpa + gpi - 1) / gpi);
    const int items1 = (int)(((long long)(na - ny) * gpa + gpi - 1) / gpi);
    const int n_items = items0 + items1;
    const int ipb = (n_items + sms - 1) / sms;
    const Layout L = layout_for(n, na, nb, P, n_items);
    if (L.total > kStaticScratchBytes) {
        set_msg(err, err_cap,
                "n=%d, n_angles=%d, n_bins=%d need %zu bytes of scratch; the fixed scratch holds %zu "
                "(about n <= 1220 at 720 angles)",
                n, na, nb, L.total, kStaticScratchBytes);
        return MC_EINVAL;
    }

    unsigned char* b = static_cast<unsigned char*>(base);
    int* d_err = reinterpret_cast<int*>(b + L.err);
    RigidGate* d_rg = reinterpret_cast<RigidGate*>(b + L.rigid);
    FwdAngle* d_ang = reinterpret_cast<FwdAngle*>(b + L.ang);
    int2* d_groups = reinterpret_cast<int2*>(b + L.groups);
    RayItem* d_items = reinterpret_cast<RayItem*>(b + L.items);
    float2* d_lrow = reinterpret_cast<float2*>(b + L.lrow);
    float2* d_lcol = reinterpret_cast<float2*>(b + L.lcol);

    // the array keeps the previous call's contents: the error word and the
    // zero guard cells of both line layouts must start at zero
    cudaError_t e = cudaMemsetAsync(b + L.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + L.lrow, 0, L.total - L.lrow, s);
    if (e != cudaSuccess) {
        set_msg(err, err_cap, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        return MC_ECUDA;
    }
    const int tot = na + (int)n_groups + n_items + 1;
    k_static_tables<<<(tot + 255) / 256, 256, 0, s>>>(n, na, nb, lc, (int)gpi, items0, rigid ? 1 : 0,
                                                     rigid ? rigid[0] : 0.0, rigid ? rigid[1] : 0.0,
                                                     rigid ? rigid[2] : 0.0, d_ang, d_groups, d_items, d_rg);
    e = cudaGetLastError();
    WarpArgs w{};
    w.x = x; w.n = n; w.rigid = d_rg; w.field = nullptr; w.identity = rigid ? 0 : 1;
    w.sel = GateSel{nullptr, 0}; w.n_slots = 1;
    w.lrow = d_lrow; w.lcol = d_lcol; w.layout_stride = (size_t)layout_lines(n) * P; w.P = P;
    w.guard = kGuardNarrow;
    if (e == cudaSuccess) e = launch_warp_layouts(w, s);
    FwdArgs f{};
    f.lrow = d_lrow; f.lcol = d_lcol; f.layout_stride = (size_t)layout_lines(n) * P; f.P = P;
    f.guard = kGuardNarrow;
    f.ang = d_ang; f.groups = d_groups; f.items = d_items; f.n_items = n_items;
    f.ipb = ipb; f.rpt = rpt; f.lc = lc; f.n = n; f.na = na; f.nb = nb;
    f.sel = GateSel{nullptr, 0}; f.n_slots = 1; f.mode = 0; f.out = out; f.err = d_err;
    if (stall_requested()) {
        // test hook of the failure path: the producer issues no copies and the
        // consumers' waits run out after 2^12 polls, setting the error word
        f.stall = 1;
        f.wait_limit = 1u << 12;
    }
    if (e == cudaSuccess) e = launch_forward(f, s);
    if (e != cudaSuccess) {
        set_msg(err, err_cap, "kernel launch failed: %s", cudaGetErrorString(e));
        return MC_ECUDA;
    }
    return MC_OK;
}

extern "C" mc_status mc_forward_static_status(void* cuda_stream, char* err, int32_t err_cap)
{
    if (err && err_cap > 0) err[0] = '\0';
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_msg(err, err_cap, "no CUDA device");
        return MC_EDEVICE;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (dev >= 0 && dev < kMaxDevices) base = g_ptr[dev];
    }
    if (!base) {
        set_msg(err, err_cap, "mc_forward_static has not run on device %d", dev);
        return MC_ESTATE;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap_st) != cudaSuccess || cap_st != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        set_msg(err, err_cap, "the status is read outside stream capture, on a valid stream");
        return MC_EINVAL;
    }
    // the error word sits at the start of the scratch array
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, base, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_msg(err, err_cap, "reading the error word failed: %s", cudaGetErrorString(e));
        return MC_ECUDA;
    }
    if (h == kErrTimeout) {
        set_msg(err, err_cap, "a device-side wait of the projection ran out of polls; out is incomplete");
        return MC_ETIMEOUT;
    }
    if (h != kErrNone) {
        set_msg(err, err_cap, "device error word %d (out-of-bounds sample); out is incomplete", h);
        return MC_EDEVICE;
    }
    return MC_OK;
}
