// Device-side layouts, tables and helpers shared by the libmc kernels.
//
// HBM layouts (per gate slot):
//   line layouts  Two copies of the warped image w = D_i x, each as
//                 layout_lines(n) lines (n rounded up to a multiple of 8, the
//                 extra lines zero) of pitch P = layout_pitch(n, guard) float2
//                 "pairs" (w[p], w[p+1] - w[p]) with `guard` zero cells before
//                 the data and at least `guard` after it:
//                 ROWS  line l = image row l    (used by rows-driven angles),
//                 COLS  line l = image column l (used by columns-driven angles).
//                 One 8-byte load gives both interpolation taps, and the zero
//                 guards make the Joseph interpolation branch-free.
//   dy            Dual increment of one gate as n_angles lines of pitch Pb
//                 float2 pairs (m_k dy[b], m_k dy[b+1]), pre-scaled by the
//                 angle's sample step m_k, with Gb zero bins before the data,
//                 so that the pixel-driven gather reads both of its bins with
//                 one 8-byte load and no bounds checks.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace mcg {

// Zero pairs before each image line of a layout (and at least as many after
// it): the forward projector's clamped positions need 2 CL + 1 of them for
// parts of CL lines, so 17 serve parts of up to 8 lines and 33 whole 16-line
// chunks.  A context takes the wide guard where a 3-stage ring of 16-line
// chunks with such lines fits (small images); elsewhere 16-line chunks are
// sampled in two 8-line parts.
constexpr int kGuardNarrow = 17, kGuardWide = 33;
__host__ __device__ constexpr int guard_max_lines(int guard) { return (guard - 1) / 2; }

// Lines and pitch (pairs) of a line layout: whole chunks of 8 lines (16 where
// the line count allows), and a pitch P >= n + 2 guard.
__host__ __device__ constexpr int layout_lines(int n) { return (n + 7) / 8 * 8; }
__host__ __device__ constexpr int layout_pitch(int n, int guard) { return (n + 2 * guard + 3) / 4 * 4; }
// Stages of lc lines x P pairs that kRingBytes of shared memory (what a block
// has beside its static tables) holds, at most kMaxStages.
constexpr int kMaxStages = 5;
constexpr size_t kRingBytes = 221440;
__host__ __device__ constexpr int forward_stages(int lc, int P)
{
    return kRingBytes / ((size_t)lc * P * 8) < (size_t)kMaxStages ? (int)(kRingBytes / ((size_t)lc * P * 8))
                                                                  : kMaxStages;
}
// The ring a chunk size runs with (the kernels are compiled for these): five
// stages, or three for 16-line chunks and for 8-line chunks whose five stages
// do not fit (large images); 4- and 2-line chunks always fit five.
__host__ __device__ constexpr int forward_ring(int lc, int P)
{
    return lc >= 16 ? 3 : (lc == 8 && forward_stages(lc, P) < 5 ? 3 : 5);
}
// A chunk is sampled in parts of at most as many lines as the guard's clamp
// reaches (each part clamps its own starting position): whole chunks where
// the guard allows, two 8-line parts of a 16-line chunk with the narrow guard.
__host__ __device__ constexpr int forward_part_lines(int lc, int guard)
{
    return lc < guard_max_lines(guard) ? lc : guard_max_lines(guard);
}
// Whether chunks of lc lines can run on layouts of n lines and pitch P: whole
// chunks and room for their ring.
__host__ __device__ constexpr bool forward_lines_fit(int n, int P, int guard, int lc)
{
    return (lc == 2 || lc == 4 || lc == 8 || lc == 16) && guard >= 2 * 2 + 1 && layout_lines(n) % lc == 0 &&
           forward_stages(lc, P) >= forward_ring(lc, P);
}
// Consumer warps of a forward block (plus one producer warp): 23 at 80
// registers, or 15 with up to 128 registers for 16-line chunks sampled in two
// 8-line parts (measured at rigid512: the register count, not the warp count,
// paid there; other shapes kept 23).
__host__ __device__ constexpr int forward_warps(int lc, int cl) { return (lc == 16 && cl == 8) ? 15 : 23; }
// The default chunk: the longest that fits (measured SPDHG epochs: 16-line
// chunks in three stages beat 8-line ones at 128^2-384^2 with the wide guard
// and at 512^2 in two 8-line parts with the narrow one, 1.661 against 1.704
// ms; 8-line chunks in three stages beat 4-line ones in five at 768^2 and
// 1024^2).
__host__ __device__ constexpr int forward_default_lines(int n, int P, int guard)
{
    return forward_lines_fit(n, P, guard, 16) ? 16
         : forward_lines_fit(n, P, guard, 8)  ? 8
         : forward_lines_fit(n, P, guard, 4)  ? 4 : 2;
}
// The guard of a context's layouts: wide where 16-line chunks fit their ring.
__host__ __device__ constexpr int layout_guard(int n)
{
    return forward_lines_fit(n, layout_pitch(n, kGuardWide), kGuardWide, 16) ? kGuardWide : kGuardNarrow;
}
constexpr float kMagic = 12582912.0f;     // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;    // bit pattern of kMagic

// Joseph sampling table of one angle (host float64 -> float32).
// Along a line l of the driving axis the ray (k, b) sits at the padded
// position u = (b - hb) * inv - (l - h) * t + h + guard.  Between the first
// lines of two consecutive sampled parts (CL lines: a whole chunk, or half of
// a 16-line chunk) u moves by -CL * t, split exactly into step_int +
// step_frac (step_frac in [0, 1)).
struct FwdAngle {
    float t_hi;             // cos/sin or sin/cos (first 16 bytes: chunk loop)
    float step_frac;
    int step_int;
    float delta;            // |inv| = sample step length
    float inv_hi, inv_lo;   // 1/sin (columns-driven) or 1/cos (rows-driven)
    float t_lo;
    int dir;                // 1: lines are image columns, 0: image rows
};

// Pixel-driven gather table of one angle: pixel (r, c) projects to the
// detector coordinate beta = (c - h) cos + (r - h) sin + hb (+ Gb padding).
struct BpAngle {
    float cos_hi, cos_lo, sin_hi, sin_lo;
    float m;                // 1/max(|sin|, |cos|): step length, also hat slope
    float m2;               // m*m
    float cos_h19, cos_l19; // cos = cos_h19 + cos_l19 with at most 19 significant bits in
                            // cos_h19, so that l * cos_h19 is exact for 0 <= l < 32
};

// Rigid warp of one gate: q = R(phi) p + t about the image centre, stored as
// float pairs so that positions are exact to ~1e-6 px at any image size.
struct RigidGate {
    float cos_hi, cos_lo, sin_hi, sin_lo;
    float offx_hi, offx_lo, offy_hi, offy_lo;   // tx + h, ty + h
};

// One block's share of the forward rays: ray groups [begin, end) of the
// group table, all with the same driving axis.  A ray group is up to 32
// consecutive bins of one angle (one warp).
struct RayItem {
    int begin, end, dir, band;     // band: chunk band of a banded (angle-subset) item, else 0
};

// ---- programmatic dependent launch ----------------------------------------
// The kernels of an iteration are launched with programmatic stream
// serialisation (pdl_launch below): the next kernel's blocks may be scheduled
// while the previous kernel finishes.  Each such kernel first waits until its
// predecessor has completed and its writes are visible (pdl_wait), and only
// then lets its own successor be scheduled (pdl_trigger), so at most one
// kernel is waiting behind a running one.  For a kernel launched the ordinary
// way both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---- exact little helpers ------------------------------------------------
// floor(v) as float, and its integer in i (valid for |v| < 2^22): adding
// 1.5*2^23 with round-toward-minus-infinity leaves floor(v) in the mantissa.
__device__ __forceinline__ float floor_magic(float v, int& i)
{
    const float t = __fadd_rd(v, kMagic);
    i = __float_as_int(t) - kMagicBits;
    return __fsub_rn(t, kMagic);
}

// Error-free sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// x * (yhi + ylo) as a float pair (x exactly representable, |x| < 2^12).
__device__ __forceinline__ void mul_df(float x, float yhi, float ylo, float& hi, float& lo)
{
    hi = __fmul_rn(x, yhi);
    lo = fmaf(x, ylo, fmaf(x, yhi, -hi));
}

// Split hi + lo (|lo| << 1) into an integer part and a fraction in [0, 1).
__device__ __forceinline__ void split_int_frac(float hi, float lo, int& ip, float& frac)
{
    const float f = floorf(hi);
    ip = (int)f;
    frac = __fadd_rn(__fsub_rn(hi, f), lo);
    if (frac < 0.0f) { frac = __fadd_rn(frac, 1.0f); ip -= 1; }
    else if (frac >= 1.0f) { frac = __fsub_rn(frac, 1.0f); ip += 1; }
}

// Bilinear taps of the pull-back warp at output pixel (r, c): top-left
// source pixel (r0, c0) and fractions (fr, fc).  Rigid positions are
// computed in float-pair arithmetic; dense fields split u into integer and
// fraction exactly.  K1 (warp) and K2 (transpose CSR) both call this, so
// D_i^T is the exact transpose of D_i.
__device__ __forceinline__ void warp_taps(const RigidGate* rg, const float* field, int n,
                                          int r, int c, int& r0, int& c0, float& fr, float& fc)
{
    if (field) {
        const size_t p = (size_t)r * n + c;
        const float ux = field[p], uy = field[(size_t)n * n + p];
        const float fx = floorf(ux), fy = floorf(uy);
        c0 = c + (int)fx; fc = __fsub_rn(ux, fx);
        r0 = r + (int)fy; fr = __fsub_rn(uy, fy);
    } else {
        const float h = 0.5f * (float)(n - 1);
        const float X = (float)c - h, Y = (float)r - h;    // exact
        float a_hi, a_lo, b_hi, b_lo, s, e, s2, e2;
        // column: X cos - Y sin + (tx + h)
        mul_df(X, rg->cos_hi, rg->cos_lo, a_hi, a_lo);
        mul_df(-Y, rg->sin_hi, rg->sin_lo, b_hi, b_lo);
        two_sum(a_hi, b_hi, s, e);
        two_sum(s, rg->offx_hi, s2, e2);
        split_int_frac(s2, ((a_lo + b_lo) + (e + e2)) + rg->offx_lo, c0, fc);
        // row: X sin + Y cos + (ty + h)
        mul_df(X, rg->sin_hi, rg->sin_lo, a_hi, a_lo);
        mul_df(Y, rg->cos_hi, rg->cos_lo, b_hi, b_lo);
        two_sum(a_hi, b_hi, s, e);
        two_sum(s, rg->offy_hi, s2, e2);
        split_int_frac(s2, ((a_lo + b_lo) + (e + e2)) + rg->offy_lo, r0, fr);
    }
}

// ---- reduced-precision storage of d and y (1: binary16, 2: bfloat16) --------
__device__ __forceinline__ float load_store(unsigned short v, int store)
{
    return store == 1 ? __half2float(__ushort_as_half(v)) : __bfloat162float(__ushort_as_bfloat16(v));
}

__device__ __forceinline__ unsigned short to_store(float v, int store)
{
    return store == 1 ? __half_as_ushort(__float2half_rn(v)) : __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// ---- Philox4x32-10 (Salmon et al., SC'11) ----------------------------------
__device__ __forceinline__ uint32_t philox_word0(uint64_t seed, uint32_t stream, uint64_t k)
{
    uint32_t c0 = (uint32_t)k, c1 = stream, c2 = (uint32_t)(k >> 32), c3 = 0u;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return c0;
}

// ---- error word ----------------------------------------------------------
enum : int { kErrNone = 0, kErrTimeout = 1, kErrBounds = 2 };

}  // namespace mcg
