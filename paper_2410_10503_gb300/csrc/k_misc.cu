// K8 device gate draw (Algorithm 1 step (ii), serial uniform sampling
// p_i = 1/N), K9 float64 reductions (Theorem norms, objective O(x) of
// Sec. II-A, saddle-point distance), and small vector kernels.
#include <algorithm>
#include <cmath>

#include "mc_kernels.h"

namespace mcg {

namespace {

// One block.  kctr != null: k0 = *kctr and the counter advances by count
// after every thread has read it (graph replays draw fresh gates).
// thr == null: uniform, gate = floor(word0 * N / 2^32).  Otherwise serial
// sampling with P(i) = p_i: gate = the first i with word0 < thr[i], where
// thr[i] = floor(2^32 (p_0 + ... + p_i)) and thr[N-1] = 2^32.
__global__ void k_draw_gates(uint64_t seed, uint32_t stream, unsigned long long* kctr,
                             uint64_t k0_in, int count, int n_gates, const unsigned long long* thr,
                             int* out)
{
    pdl_wait();
    pdl_trigger();
    const uint64_t k0 = kctr ? (uint64_t)*kctr : k0_in;
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
        const uint32_t w = philox_word0(seed, stream, k0 + (uint64_t)j);
        int g;
        if (!thr) {
            g = (int)(((uint64_t)w * (uint64_t)n_gates) >> 32);
        } else {
            g = 0;
            while (g < n_gates - 1 && (unsigned long long)w >= thr[g]) ++g;
        }
        out[j] = g;
    }
    __syncthreads();
    if (kctr && threadIdx.x == 0) *kctr = (unsigned long long)(k0 + (uint64_t)count);
}

// dy pairs (m_k y[b], m_k y[b+1]) of one sinogram; y[nb] = 0
__global__ void k_pad_sino(const float* __restrict__ y, float2* dy, const BpAngle* ang, int na,
                           int nb, int Pb, int Gb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x - 1;
    const int k = blockIdx.y;
    if (b >= nb) return;
    const float m = ang[k].m;
    const float v0 = (b >= 0) ? m * y[(size_t)k * nb + b] : 0.0f;
    const float v1 = (b + 1 < nb) ? m * y[(size_t)k * nb + b + 1] : 0.0f;
    dy[(size_t)k * Pb + Gb + b] = make_float2(v0, v1);
}

constexpr int kRedThreads = 256;
constexpr int kRedParts = 1024;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sm[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = (lane < kRedThreads / 32) ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;   // valid in thread 0
}

// Fixed grid (kRedParts blocks) and fixed orders: bitwise reproducible.
__global__ void __launch_bounds__(kRedThreads) k_reduce(const float* __restrict__ a,
                                                        const float* __restrict__ b, size_t len,
                                                        int mode, double* partial)
{
    double acc = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const double x = (double)a[i];
        if (mode == kRedSumSq) acc += x * x;
        else if (mode == kRedDiffSq) { const double d = x - (double)b[i]; acc += d * d; }
        else acc += x * (double)b[i];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_final(const double* partial, int parts, double* out)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < parts; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void k_axpby(float a, const float* __restrict__ x, float b, const float* __restrict__ y,
                        float* out, size_t len)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] = y ? fmaf(a, x[i], b * y[i]) : a * x[i];
}

__global__ void k_normalize(float* x, const double* norm2, size_t len)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double nn = *norm2;
    const float s = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.0f;
    if (i < len) x[i] *= s;
}

__global__ void k_trace_combine(const double* dx2, const double* xs2, const double* dy2, double* out)
{
    out[0] = (*xs2 > 0.0) ? sqrt(*dx2 / *xs2) : nan("");
    out[1] = dy2 ? (*dx2 + *dy2) : nan("");
}

__global__ void k_objective_combine(const double* xx, const double* res, int n_res, double alpha,
                                    int N, double* out)
{
    double s = 0.0;
    for (int i = 0; i < n_res; ++i) s += res[i];
    *out = alpha * (*xx) + s / (double)N;
}

// Conjugate-gradient updates with the scalars kept on the device (float64):
// step 1: a = rr / pq, x += a p, r -= a q;  step 2: beta = rr_new / rr, p = r + beta p.
__global__ void k_cg_step1(float* x, float* r, const float* p, const float* q, size_t len,
                           const double* rr, const double* pq)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double den = *pq;
    const float a = den != 0.0 ? (float)(*rr / den) : 0.0f;
    if (i < len) {
        x[i] = fmaf(a, p[i], x[i]);
        r[i] = fmaf(-a, q[i], r[i]);
    }
}

__global__ void k_cg_step2(float* p, const float* r, size_t len, const double* rr_new, const double* rr_old)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double den = *rr_old;
    const float beta = den != 0.0 ? (float)(*rr_new / den) : 0.0f;
    if (i < len) p[i] = fmaf(beta, p[i], r[i]);
}

__global__ void k_fill_nan(double* p, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = nan("");
}

}  // namespace

cudaError_t launch_draw_gates(uint64_t seed, uint32_t stream, unsigned long long* kctr,
                              uint64_t k0, int count, int n_gates, const unsigned long long* thr, int* out,
                              cudaStream_t s)
{
    return pdl_launch(k_draw_gates, dim3(1), dim3(256), 0, s, seed, stream, kctr, k0, count, n_gates, thr,
                      out);
}

cudaError_t launch_pad_sino(const float* y, float2* dy, const BpAngle* ang, int na, int nb,
                            int Pb, int Gb, cudaStream_t s)
{
    const dim3 grid((nb + 1 + 255) / 256, na);
    k_pad_sino<<<grid, 256, 0, s>>>(y, dy, ang, na, nb, Pb, Gb);
    return cudaGetLastError();
}

int reduce_parts() { return kRedParts; }

cudaError_t launch_reduce(const float* a, const float* b, size_t len, int mode,
                          double* partial, double* out, cudaStream_t s)
{
    k_reduce<<<kRedParts, kRedThreads, 0, s>>>(a, b, len, mode, partial);
    k_reduce_final<<<1, kRedThreads, 0, s>>>(partial, kRedParts, out);
    return cudaGetLastError();
}

cudaError_t launch_axpby(float a, const float* x, float b, const float* y, float* out,
                         size_t len, cudaStream_t s)
{
    k_axpby<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(a, x, b, y, out, len);
    return cudaGetLastError();
}

cudaError_t launch_normalize(float* x, const double* norm2, size_t len, cudaStream_t s)
{
    k_normalize<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(x, norm2, len);
    return cudaGetLastError();
}

cudaError_t launch_trace_combine(const double* dx2, const double* xs2, const double* dy2,
                                 double* out, cudaStream_t s)
{
    k_trace_combine<<<1, 1, 0, s>>>(dx2, xs2, dy2, out);
    return cudaGetLastError();
}

cudaError_t launch_objective_combine(const double* xx, const double* res, int n_res,
                                     double alpha, int N, double* out, cudaStream_t s)
{
    k_objective_combine<<<1, 1, 0, s>>>(xx, res, n_res, alpha, N, out);
    return cudaGetLastError();
}

cudaError_t launch_cg_step1(float* x, float* r, const float* p, const float* q, size_t len,
                            const double* rr, const double* pq, cudaStream_t s)
{
    k_cg_step1<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(x, r, p, q, len, rr, pq);
    return cudaGetLastError();
}

cudaError_t launch_cg_step2(float* p, const float* r, size_t len, const double* rr_new,
                            const double* rr_old, cudaStream_t s)
{
    k_cg_step2<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(p, r, len, rr_new, rr_old);
    return cudaGetLastError();
}

// Zero up to kZeroSegs buffers in one launch (the solver-state reset):
// 16-byte stores where a segment allows them, a byte tail otherwise.
__global__ void __launch_bounds__(256) k_zero_segments(ZeroSegs z)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = 0; k < z.count; ++k) {
        unsigned char* p = static_cast<unsigned char*>(z.ptr[k]);
        const size_t bytes = z.bytes[k];
        const size_t n16 = ((uintptr_t)p & 15) ? 0 : bytes / 16;
        for (size_t i = t0; i < n16; i += stride) reinterpret_cast<uint4*>(p)[i] = make_uint4(0, 0, 0, 0);
        for (size_t i = n16 * 16 + t0; i < bytes; i += stride) p[i] = 0;
    }
}

cudaError_t launch_zero_segments(const ZeroSegs& z, cudaStream_t s)
{
    size_t tot = 0;
    for (int k = 0; k < z.count; ++k) tot += z.bytes[k];
    const int blocks = (int)std::min<size_t>(4096, std::max<size_t>(1, (tot / 16 + 255) / 256));
    k_zero_segments<<<blocks, 256, 0, s>>>(z);
    return cudaGetLastError();
}

cudaError_t launch_fill_nan(double* p, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_fill_nan<<<(count + 255) / 256, 256, 0, s>>>(p, count);
    return cudaGetLastError();
}

// ---- storage conversions ------------------------------------------------------
__global__ void k_to_store(const float* __restrict__ src, unsigned short* __restrict__ dst, size_t len,
                           int store)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = to_store(src[i], store);
}

__global__ void k_from_store(const unsigned short* __restrict__ src, float* __restrict__ dst, size_t len,
                             int store)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = load_store(src[i], store);
}

cudaError_t launch_to_store(const float* src, unsigned short* dst, size_t len, int store, cudaStream_t s)
{
    if (store != 1 && store != 2) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)std::min<size_t>((len + 255) / 256, 4096);
    k_to_store<<<std::max(blocks, 1u), 256, 0, s>>>(src, dst, len, store);
    return cudaGetLastError();
}

cudaError_t launch_from_store(const unsigned short* src, float* dst, size_t len, int store, cudaStream_t s)
{
    if (store != 1 && store != 2) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)std::min<size_t>((len + 255) / 256, 4096);
    k_from_store<<<std::max(blocks, 1u), 256, 0, s>>>(src, dst, len, store);
    return cudaGetLastError();
}

}  // namespace mcg
