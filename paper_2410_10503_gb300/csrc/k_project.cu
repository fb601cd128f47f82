// K3 Joseph forward projection A w, ray-driven, with the dual update of
// Algorithm 1 step (ii) fused into its epilogue (arXiv 2410.10503, Sec. II-A
// and Algorithm 1: y_i^{k+1} = prox_{sigma f_i^*}(y_i^k + sigma A_i x^{k+1})).
//
// Each block owns up to 256*RPT rays that share a driving axis and streams
// the whole warped image through shared memory in chunks of `lc` lines:
// one bulk TMA copy (cp.async.bulk) per chunk, two stages, mbarrier
// completion.  Every ray then samples the chunk's lines from shared memory.
// Sample positions are carried as an integer plus a float fraction relative
// to the chunk's first line (float-pair base per ray and chunk), so the
// interpolation weights are exact to ~1e-6 px whatever the image size.
#include "mc_kernels.h"

namespace mcg {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase; false after `limit` failed polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(bar, bytes);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

constexpr uint32_t kWaitLimit = 1u << 24;   // polls before a stage wait gives up
constexpr int kThreads = 256;

__device__ __forceinline__ int gate_of(const GateSel& s, int slot)
{
    return s.list ? s.list[slot] : (s.fixed >= 0 ? s.fixed : slot);
}

template <int RPT>
__global__ void __launch_bounds__(kThreads) k_forward(FwdArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* s_flag = reinterpret_cast<int*>(smem + 16);
    float* stage0 = reinterpret_cast<float*>(smem + 128);
    const size_t stage_floats = (size_t)a.lc * a.P;

    const RayItem item = a.items[blockIdx.x];
    const int slot = blockIdx.y;
    const int gate = gate_of(a.sel, slot);
    const float* src = (item.dir ? a.lcol : a.lrow) + slot * a.layout_stride;
    const int n = a.n, nb = a.nb;
    const float h = 0.5f * (float)(n - 1);
    const float hb = 0.5f * (float)(nb - 1);
    const float off = h + (float)kGuard;

    // ---- ray setup ----------------------------------------------------------
    float pbh[RPT], pbl[RPT], th[RPT], tl[RPT], acc[RPT];
    int lo[RPT], hi[RPT], kk[RPT], bb[RPT];
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        const int rho = item.begin + m * kThreads + (int)threadIdx.x;
        acc[m] = 0.0f;
        lo[m] = 1; hi[m] = 0; kk[m] = -1; bb[m] = 0;
        pbh[m] = pbl[m] = th[m] = tl[m] = 0.0f;
        if (rho < item.end) {
            const int o = rho / nb;
            const int b = rho - o * nb;
            const int k = __ldg(a.order + o);
            const FwdAngle T = a.ang[k];
            kk[m] = k; bb[m] = b;
            th[m] = T.t_hi; tl[m] = T.t_lo;
            const float B = (float)b - hb;                 // exact
            float ph, pl, s, e;
            mul_df(B, T.inv_hi, T.inv_lo, ph, pl);
            two_sum(ph, off, s, e);
            pbh[m] = s; pbl[m] = pl + e;                   // B*inv + h + guard
            // position at line 0 is pbh + h*t; lines with a non-zero weight
            // have u in (kGuard - 1, kGuard + n); widen by up to two lines
            const float u0 = fmaf(h, T.t_hi, s);
            const float t = T.t_hi;
            if (fabsf(t) < 1e-6f) {
                if (u0 > (float)kGuard - 2.0f && u0 < (float)(kGuard + n) + 1.0f) { lo[m] = 0; hi[m] = n - 1; }
            } else {
                const float e1 = (u0 - (float)(kGuard + n)) / t;
                const float e2 = (u0 - (float)(kGuard - 1)) / t;
                float l_lo = floorf(fminf(e1, e2)) - 1.0f;
                float l_hi = ceilf(fmaxf(e1, e2)) + 1.0f;
                l_lo = fmaxf(l_lo, 0.0f);
                l_hi = fminf(l_hi, (float)(n - 1));
                if (l_lo <= l_hi) { lo[m] = (int)l_lo; hi[m] = (int)l_hi; }
            }
        }
    }

    // ---- staged sweep over the image lines ---------------------------------
    const int nch = (n + a.lc - 1) / a.lc;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *s_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 2 && c < nch; ++c) {
            const int l0 = c * a.lc;
            const int lines = min(a.lc, n - l0);
            bulk_load(stage0 + c * stage_floats, src + (size_t)l0 * a.P,
                      (uint32_t)(lines * a.P * sizeof(float)), &bar[c]);
        }
    }
    bool ok = true;
    for (int ch = 0; ch < nch; ++ch) {
        const int st = ch & 1;
        if (!mbar_wait(&bar[st], (uint32_t)((ch >> 1) & 1), kWaitLimit)) {
            ok = false;
            *s_flag = 1;
        }
        __syncthreads();
        if (*s_flag) { ok = false; break; }
        const float* sb = stage0 + st * stage_floats;
        const int l0 = ch * a.lc;
        const int lines = min(a.lc, n - l0);
        const float L0 = (float)l0 - h;                      // exact
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int jlo = max(lo[m] - l0, 0);
            const int jhi = min(hi[m] - l0, lines - 1);
            if (jlo > jhi) continue;
            float qh, ql, s, e;
            mul_df(L0, th[m], tl[m], qh, ql);
            two_sum(pbh[m], -qh, s, e);
            int ui;
            float frac;
            split_int_frac(s, (pbl[m] - ql) + e, ui, frac);
            const float* base = sb + ui;
            const float t = th[m];
            float a_m = acc[m];
            float jf = (float)jlo;
            for (int j = jlo; j <= jhi; ++j, jf += 1.0f) {
                const float w = fmaf(-jf, t, frac);
                int fi;
                const float fl = floor_magic(w, fi);
                const float f = w - fl;
                const float* q = base + j * a.P + fi;
#ifdef MC_CHECKED
                const long off_q = (long)(q - sb);
                if (off_q < (long)j * a.P || off_q + 1 >= (long)(j + 1) * a.P) {
                    atomicExch(a.err, kErrBounds);
                    continue;
                }
#endif
                const float v0 = q[0], v1 = q[1];
                a_m += fmaf(f, v1 - v0, v0);
            }
            acc[m] = a_m;
        }
        __syncthreads();
        if (threadIdx.x == 0 && ch + 2 < nch) {
            const int l2 = (ch + 2) * a.lc;
            const int lines2 = min(a.lc, n - l2);
            bulk_load(stage0 + st * stage_floats, src + (size_t)l2 * a.P,
                      (uint32_t)(lines2 * a.P * sizeof(float)), &bar[st]);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(a.err, kErrTimeout);
            // give copies still in flight a bounded chance to land
            for (int c = 0; c < 2; ++c) mbar_wait(&bar[c], 0u, 1u << 16);
        }
        return;
    }

    // ---- epilogue -------------------------------------------------------------
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        if (kk[m] < 0) continue;
        const int k = kk[m], b = bb[m];
        const float val = a.ang[k].delta * acc[m];
        const size_t idx = (size_t)k * nb + b;
        if (a.mode == 0) {
            a.out[(size_t)slot * a.na * nb + idx] = val;
        } else {
            const size_t gi = (size_t)gate * a.na * nb + idx;
            const float yo = a.y[gi];
            const float yn = (yo + a.sigma * (val - a.d[gi])) * a.inv_den;
            a.y[gi] = yn;
            a.dy[slot * a.dy_stride + (size_t)k * a.Pb + a.Gb + b] = yn - yo;
        }
    }
}

}  // namespace

size_t forward_smem_bytes(int lc, int P) { return 128 + 2 * (size_t)lc * P * sizeof(float); }

cudaError_t forward_prepare(int max_smem)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_forward<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_forward<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_forward<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_forward<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    return cudaSuccess;
}

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s)
{
    const dim3 grid(a.n_items, a.n_slots);
    const size_t smem = forward_smem_bytes(a.lc, a.P);
    switch (a.rpt) {
    case 1: k_forward<1><<<grid, kThreads, smem, s>>>(a); break;
    case 2: k_forward<2><<<grid, kThreads, smem, s>>>(a); break;
    case 4: k_forward<4><<<grid, kThreads, smem, s>>>(a); break;
    case 8: k_forward<8><<<grid, kThreads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mcg
