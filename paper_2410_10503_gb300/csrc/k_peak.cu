// Shared-memory load bandwidth of this GPU, the denominator of the
// projectors' roofline: both Joseph projectors (A and its matched adjoint,
// Sec. II-A) gather 8-byte pairs from shared memory, so their bound is the
// rate at which the SMs deliver conflict-free 64-bit shared loads.
//
// Every warp streams 64-bit shared loads (ld.shared.b64, the width of the
// projectors' ld.shared.v2.f32) over a 32 KB buffer at consecutive
// 8-byte addresses (a warp's 256 bytes cover all 32 banks twice: two
// wavefronts, no conflict), and packs the loaded pairs into one add.f32x2 per
// load so that the loads cannot be dropped and issue stays far below the
// load pipe's rate.  Two blocks of 1024 threads per SM keep all of them
// resident at once; each block records its clock64 span, so the result is
// given both per second (CUDA events) and per SM clock.
#include <algorithm>
#include <vector>

#include "mc.h"
#include "mc_kernels.h"

namespace {

constexpr int kPeakThreads = 1024;
constexpr int kPeakBytes = 32768;                  // shared buffer per block
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads, 2) k_smem_peak(int reps, float* sink, long long* cycles)
{
    __shared__ __align__(16) float2 buf[kPeakBytes / 8];
    for (int i = threadIdx.x; i < kPeakBytes / 8; i += blockDim.x)
        buf[i] = make_float2((float)i, 1.0f);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    // warp w starts at its own 256-byte row; each step moves every warp on by
    // one row (wrapping inside the buffer), lanes at consecutive pairs
    uint32_t off = (uint32_t)(warp * 256);
    unsigned long long acc;
    asm volatile("mov.b64 %0, 0;" : "=l"(acc));
    __syncthreads();
    const long long t0 = clock64();
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
            const uint32_t a = base + ((off + (uint32_t)(u * 256)) & (kPeakBytes - 1)) + lane * 8;
            unsigned long long v;
            asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
            asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(acc) : "l"(v));
        }
        off += (uint32_t)(kPeakUnroll * 256);
    }
    __syncthreads();
    const long long t1 = clock64();
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc));
    if (lo + hi == -1.0f) sink[blockIdx.x] = lo;   // never true; keeps the loads
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" mc_status mc_measure_shared_load_peak(int32_t reps, double* out)
{
    if (!out || reps < 1) return MC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MC_EDEVICE; }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) return MC_EDEVICE;
    const int blocks = 2 * sms;
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    mc_status st = MC_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && st == MC_OK) st = MC_ECUDA;
        return e == cudaSuccess;
    };
    if (ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) && ck(cudaMalloc(&sink, blocks * sizeof(float))) &&
        ck(cudaMalloc(&cyc, blocks * sizeof(long long))) && ck(cudaEventCreate(&e0)) && ck(cudaEventCreate(&e1))) {
        const int inner = 128;                             // 16 KB per thread per rep: ~5 GB per rep
        // warm-up, then the timed launch
        k_smem_peak<<<blocks, kPeakThreads, 0, s>>>(inner, sink, cyc);
        ck(cudaGetLastError());
        ck(cudaEventRecord(e0, s));
        k_smem_peak<<<blocks, kPeakThreads, 0, s>>>(inner * reps, sink, cyc);
        ck(cudaGetLastError());
        ck(cudaEventRecord(e1, s));
        float ms = 0.0f;
        std::vector<long long> h(blocks);
        if (ck(cudaEventSynchronize(e1)) && ck(cudaEventElapsedTime(&ms, e0, e1)) &&
            ck(cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost))) {
            const double bytes = (double)blocks * kPeakThreads * (double)inner * reps * kPeakUnroll * 8.0;
            std::sort(h.begin(), h.end());
            const double cyc_max = (double)h.back();
            out[0] = bytes / (ms * 1e-3);                  // bytes per second, whole GPU
            out[1] = bytes / sms / cyc_max;                // bytes per SM clock
            out[2] = cyc_max / (ms * 1e-3) * 1e-9;         // SM clock seen by the kernel (GHz)
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (s) cudaStreamDestroy(s);
    return st;
}
