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
// resident at once; each block records its clock64 start and end and its SM,
// so the result is given both per second (CUDA events) and per SM clock (an
// SM's blocks' loads over the span of that SM's clock they covered).
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
    if (threadIdx.x == 0) {
        unsigned smid;
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        cycles[3 * blockIdx.x] = t0;                // the SM's own clock: compared only
        cycles[3 * blockIdx.x + 1] = t1;            // with blocks on the same SM
        cycles[3 * blockIdx.x + 2] = smid;
    }
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
        ck(cudaMalloc(&cyc, 3 * blocks * sizeof(long long))) && ck(cudaEventCreate(&e0)) && ck(cudaEventCreate(&e1))) {
        const int inner = 128;                             // 16 KB per thread per rep: ~5 GB per rep
        // warm-up, then the timed launch
        k_smem_peak<<<blocks, kPeakThreads, 0, s>>>(inner, sink, cyc);
        ck(cudaGetLastError());
        ck(cudaEventRecord(e0, s));
        k_smem_peak<<<blocks, kPeakThreads, 0, s>>>(inner * reps, sink, cyc);
        ck(cudaGetLastError());
        ck(cudaEventRecord(e1, s));
        float ms = 0.0f;
        std::vector<long long> h(3 * (size_t)blocks);
        if (ck(cudaEventSynchronize(e1)) && ck(cudaEventElapsedTime(&ms, e0, e1)) &&
            ck(cudaMemcpy(h.data(), cyc, 3 * blocks * sizeof(long long), cudaMemcpyDeviceToHost))) {
            const double per_block = (double)kPeakThreads * (double)inner * reps * kPeakUnroll * 8.0;
            const double bytes = (double)blocks * per_block;
            // per SM: its blocks' loads over the span from the first start to
            // the last end on that SM's clock
            std::vector<long long> lo(sms, -1), hi(sms, -1);
            std::vector<int> nblk(sms, 0);
            for (int b = 0; b < blocks; ++b) {
                const long long smid = h[3 * (size_t)b + 2];
                if (smid < 0 || smid >= sms) continue;
                const long long t0 = h[3 * (size_t)b], t1 = h[3 * (size_t)b + 1];
                lo[smid] = lo[smid] < 0 ? t0 : std::min(lo[smid], t0);
                hi[smid] = std::max(hi[smid], t1);
                ++nblk[smid];
            }
            double b_sum = 0.0, c_sum = 0.0;
            for (int m = 0; m < sms; ++m)
                if (nblk[m] > 0 && hi[m] > lo[m]) {
                    b_sum += nblk[m] * per_block;
                    c_sum += (double)(hi[m] - lo[m]);
                }
            const int used = (int)std::count_if(nblk.begin(), nblk.end(), [](int v) { return v > 0; });
            out[0] = bytes / (ms * 1e-3);                               // bytes per second, whole GPU
            out[1] = c_sum > 0 ? b_sum / c_sum : 0.0;                   // bytes per SM clock
            out[2] = used > 0 ? c_sum / used / (ms * 1e-3) * 1e-9 : 0.0; // mean SM span over event time (GHz)
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (s) cudaStreamDestroy(s);
    return st;
}
