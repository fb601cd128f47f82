// K4 pixel-driven gather backprojection A^T dy (arXiv 2410.10503, Algorithm 1
// step (iii) applies A_i^* = D_i^T A^T to the dual increment).
//
// The forward projector gives ray (k, b) the weight Delta_k * hat(u - p) on
// pixel p of driving line l, where u is the ray's position on that line and
// hat(t) = max(0, 1 - |t|).  As a function of the bin, u - p = (b - beta) * inv_k
// with beta the detector coordinate of the pixel centre, so pixel (r, c)
// collects from exactly two bins per angle, floor(beta) and floor(beta) + 1,
// with weights m * max(0, 1 - d m) and m * max(0, 1 - (1 - d) m), d = frac(beta),
// m = |inv_k| = Delta_k.  This is the transpose of the forward matrix; no
// atomics, every pixel is written once.
//
// Each thread owns PJ consecutive rows of one column.  Per angle it forms
// beta of its first pixel in float-pair arithmetic (integer bin + fraction)
// and steps the fraction by sin(phi) down the column, so d is exact to ~1e-6.
#include "mc_kernels.h"

namespace mcg {

namespace {

constexpr int kAngChunk = 256;   // angle-table entries staged in shared memory

template <int PJ>
__global__ void __launch_bounds__(256) k_backproject(BpArgs a)
{
    __shared__ BpAngle s_ang[kAngChunk];
    const int n = a.n;
    const int slot = blockIdx.z;
    const int c = blockIdx.x * 32 + (int)threadIdx.x;
    const int r0 = (blockIdx.y * 8 + (int)threadIdx.y) * PJ;
    const int cc = min(c, n - 1);
    const float h = 0.5f * (float)(n - 1);
    const float X = (float)cc - h;                 // exact
    const float Y0 = (float)r0 - h;                // exact
    const float offb = 0.5f * (float)(a.nb - 1) + (float)a.Gb;
    const float* dys = a.dy + slot * a.dy_stride;

    float acc[PJ];
#pragma unroll
    for (int j = 0; j < PJ; ++j) acc[j] = 0.0f;

    // warps whose rows all lie below the image only help stage the tables
    const bool active = r0 < n;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    for (int k0 = 0; k0 < a.na; k0 += kAngChunk) {
        const int cnt = min(kAngChunk, a.na - k0);
        __syncthreads();
        for (int i = tid; i < cnt; i += 256) s_ang[i] = a.ang[k0 + i];
        __syncthreads();
        for (int i = 0; active && i < cnt; ++i) {
            const BpAngle T = s_ang[i];
            float ah, al, bh, bl, s, e, s2, e2;
            mul_df(X, T.cos_hi, T.cos_lo, ah, al);
            mul_df(Y0, T.sin_hi, T.sin_lo, bh, bl);
            two_sum(ah, bh, s, e);
            two_sum(s, offb, s2, e2);
            int bi;
            float frac;
            split_int_frac(s2, (al + bl) + (e + e2), bi, frac);
            const float* row = dys + (size_t)(k0 + i) * a.Pb + bi;
            const float m = T.m, m2 = T.m2, mm = T.m - T.m2;
#pragma unroll
            for (int j = 0; j < PJ; ++j) {
                const float beta = fmaf((float)j, T.sin_hi, frac);
                int fi;
                const float fb = floor_magic(beta, fi);
                const float d = beta - fb;
                const float w0 = fmaxf(0.0f, fmaf(-d, m2, m));
                const float w1 = fmaxf(0.0f, fmaf(d, m2, mm));
                const float y0 = __ldg(row + fi), y1 = __ldg(row + fi + 1);
                acc[j] = fmaf(w0, y0, fmaf(w1, y1, acc[j]));
            }
        }
    }
    if (c < n) {
#pragma unroll
        for (int j = 0; j < PJ; ++j) {
            const int r = r0 + j;
            if (r < n) a.out[(size_t)slot * n * n + (size_t)r * n + c] = acc[j];
        }
    }
}

}  // namespace

cudaError_t launch_backproject(const BpArgs& a, cudaStream_t s)
{
    const int rows_per_block = 8 * a.pj;
    const dim3 grid((a.n + 31) / 32, (a.n + rows_per_block - 1) / rows_per_block, a.n_slots);
    const dim3 block(32, 8);
    switch (a.pj) {
    case 4: k_backproject<4><<<grid, block, 0, s>>>(a); break;
    case 8: k_backproject<8><<<grid, block, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mcg
