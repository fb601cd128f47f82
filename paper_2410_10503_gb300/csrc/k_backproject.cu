// K4 pixel-driven gather backprojection A^T dy (arXiv 2410.10503, Algorithm 1
// step (iii) applies A_i^* = D_i^T A^T to the dual increment).
//
// The forward projector gives ray (k, b) the weight Delta_k * hat(u - p) on
// pixel p of driving line l, where u is the ray's position on that line and
// hat(t) = max(0, 1 - |t|).  As a function of the bin, u - p = (b - beta) * inv_k
// with beta the detector coordinate of the pixel centre, so pixel (r, c)
// collects from exactly two bins per angle, floor(beta) and floor(beta) + 1,
// with weights m * sat(1 - d m) and m * sat(1 - (1 - d) m), d = frac(beta),
// m = |inv_k| = Delta_k.  This is the transpose of the forward matrix; no
// atomics, every pixel is written once.  The dual increment arrives as pairs
// (m dy[b], m dy[b+1]) so one 8-byte load feeds both weights.
//
// A block owns a tile of 32 columns x PJ rows; its 8 warps all cover that
// tile, each for every 8th angle, and their partial sums are added in a fixed
// order through shared memory at the end.  Each warp runs its own staging
// pipeline: for a batch of kBatch of its angles, lanes 0..kBatch-1 each issue
// one bulk TMA copy of the window of dy pairs that the tile projects onto (WL
// pairs) into the warp's half of a two-batch ring, completed on the warp's
// mbarrier, and store the angle's constants beside it.  The next batch is in
// flight while the warp gathers from the current one, and no warp waits for
// another until the final sum, so the gathers are shared-memory loads whose
// lanes (consecutive columns, |cos| <= 1 bin apart) rarely share a bank.
//
// Positions: the staging lane forms beta at the tile's first pixel in
// float-pair arithmetic (integer bin + fraction f0); column c0 + l adds
// l cos, split on the host as cos_h19 + cos_l19 with l cos_h19 exact, so a
// lane's fraction costs two FMAs and a floor and is within ~2e-6 of exact.
// A thread owns PJ consecutive rows of one column and steps the fraction by
// sin(phi) down the column, two rows at a time in paired FP32 arithmetic.
#include <algorithm>
#include <cmath>

#include "mc_kernels.h"

namespace mcg {

namespace {

constexpr int kGroups = 8;       // warps per block = interleaved angle groups
constexpr int kBatch = 8;        // angles per staged batch of one warp
constexpr int kRing = 2;         // batches per warp in shared memory
constexpr uint32_t kWaitLimit = 1u << 24;

// Constants of one staged angle, next to its window (two 16-byte loads; the
// first pair of words is the packed row step).
struct __align__(16) AngSlot {
    float sin0, sin1;            // sin(phi) twice
    float cos_h, cos_l;          // cos(phi) = cos_h + cos_l, l * cos_h exact
    float m, om;                 // hat slope m and 1 - m
    float f0;                    // fraction of beta at the tile's first pixel
    int off;                     // window pair of beta's integer part there, plus slot * WL
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

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

// Stage one batch of the calling warp's angles: lane i < cnt takes the
// warp's angle q0 + i, i.e. k = sub + (g + (q0 + i) kGroups) S, forms beta of
// the tile's first pixel (X0, Y0), stores the angle's constants and issues
// the copy of its window: WL pairs of dy row k from ws (even, so the copy is
// 16-byte aligned), covering every bin the tile's pixels project onto.
__device__ __forceinline__ void issue_batch(const BpArgs& a, const float2* dys, int sub, int S, int g, int q0,
                                            int cnt, int wl, float X0, float Y0, float xmax, float ymax,
                                            float2* win, AngSlot* slots, uint64_t* bar)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"((uint32_t)(cnt * wl * sizeof(float2)))
                     : "memory");
    }
    __syncwarp();
    if (lane < cnt) {
        const int k = sub + (g + (q0 + lane) * kGroups) * S;
        const BpAngle T = a.ang[k];
        const float offb = 0.5f * (float)(a.nb - 1) + (float)a.Gb;
        const float b1 = fminf(X0 * T.cos_hi, xmax * T.cos_hi) + fminf(Y0 * T.sin_hi, ymax * T.sin_hi) + offb;
        int ws = ((int)floorf(b1) - 2) & ~1;
        ws = max(0, min(ws, a.Pb - wl));
        // beta(X0, Y0) = X0 cos + Y0 sin + offb as integer + fraction
        float ah, al, bh, bl, s, e, s2, e2;
        mul_df(X0, T.cos_hi, T.cos_lo, ah, al);
        mul_df(Y0, T.sin_hi, T.sin_lo, bh, bl);
        two_sum(ah, bh, s, e);
        two_sum(s, offb, s2, e2);
        int bi;
        float f0;
        split_int_frac(s2, (al + bl) + (e + e2), bi, f0);
        slots[lane] = AngSlot{T.sin_hi, T.sin_hi, T.cos_h19, T.cos_l19, T.m, 1.0f - T.m, f0,
                              lane * wl + bi - ws};
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(win + (size_t)lane * wl)),
            "l"(dys + (size_t)k * a.Pb + ws), "r"((uint32_t)(wl * sizeof(float2))), "r"(smem_u32(bar))
            : "memory");
    }
    __syncwarp();
}


__device__ __forceinline__ unsigned long long bp_pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

#ifndef MC_CHECKED
// Two rows of one column, as PTX on packed pairs: beta = j sn + frac, its
// floor through the round-down magic add (whose bits also give the window
// index), the fraction d, then the two 8-byte shared loads of the rows' dy
// pairs; jj = (j, j+1) and mm = (magic, magic) stay in registers.
__device__ __forceinline__ void bp_two_rows(unsigned long long jj, unsigned long long sn2, unsigned long long fr2,
                                            unsigned long long mm, uint32_t row, float& d0, float& d1,
                                            float2& y0, float2& y1)
{
    asm volatile(
        "{\n\t"
        ".reg .b64 b2, t2, fb2, d2;\n\t"
        ".reg .b32 q0, q1, a0, a1;\n\t"
        "fma.rn.f32x2 b2, %6, %7, %8;\n\t"
        "add.rm.f32x2 t2, b2, %9;\n\t"
        "sub.rn.f32x2 fb2, t2, %9;\n\t"
        "sub.rn.f32x2 d2, b2, fb2;\n\t"
        "mov.b64 {q0, q1}, t2;\n\t"
        "mov.b64 {%0, %1}, d2;\n\t"
        "mad.lo.u32 a0, q0, 8, %10;\n\t"
        "mad.lo.u32 a1, q1, 8, %10;\n\t"
        "ld.shared.v2.f32 {%2, %3}, [a0];\n\t"
        "ld.shared.v2.f32 {%4, %5}, [a1];\n\t"
        "}"
        : "=f"(d0), "=f"(d1), "=f"(y0.x), "=f"(y0.y), "=f"(y1.x), "=f"(y1.y)
        : "l"(jj), "l"(sn2), "l"(fr2), "l"(mm), "r"(row));
}

#endif

// pj: the rows of this launch's tiles (even, <= PJ; every caller passes PJ,
// so the row bounds below are compile-time); the register arrays are sized for
// PJ.
template <int PJ, bool SUB>
__device__ __forceinline__ void bp_block(const BpArgs& a, int bx, int by, int slot, int pj)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);                             // [kGroups][kRing]
    AngSlot* s_slot = reinterpret_cast<AngSlot*>(smem + 128);                       // [kGroups][kRing][kBatch]
    float2* s_win = reinterpret_cast<float2*>(smem + 128 + kGroups * kRing * kBatch * sizeof(AngSlot));
    const int wl = a.wl;
    const int n = a.n;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c0 = bx * 32, c = c0 + lane;
    const int r0 = by * pj;
    const float h = 0.5f * (float)(n - 1);
    const float le = (float)min(lane, n - 1 - c0);       // column offset in the tile (clamped at the edge)
    const float2* dys = a.dy + slot * a.dy_stride;
    // tile extent in centred coordinates (columns past the image are clamped)
    const float X0 = (float)c0 - h, xmax = (float)min(c0 + 31, n - 1) - h;   // exact
    const float Y0 = (float)r0 - h, ymax = Y0 + (float)(pj - 1);
    // angles of this launch: one angle subset of the drawn block, or all;
    // this warp takes the subset's angles g, g + kGroups, ...
    const int S = SUB ? a.sel.subsets : 1;
    const int sub = SUB ? sel_subset(a.sel, slot) : 0;
    const int na_s = SUB ? (a.na - sub + S - 1) / S : a.na;
    const int nq = na_s > g ? (na_s - g + kGroups - 1) / kGroups : 0;
    const int nbt = (nq + kBatch - 1) / kBatch;
    uint64_t* my_full = full + g * kRing;
    AngSlot* my_slot = s_slot + g * kRing * kBatch;
    float2* my_win = s_win + (size_t)g * kRing * kBatch * wl;

    if (lane == 0) {
        for (int i = 0; i < kRing; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&my_full[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (nbt > 0)
        issue_batch(a, dys, sub, S, g, 0, min(kBatch, nq), wl, X0, Y0, xmax, ymax, my_win, my_slot,
                    &my_full[0]);

    float acc[PJ];
#pragma unroll
    for (int j = 0; j < PJ; ++j) acc[j] = 0.0f;
    unsigned long long jj[PJ / 2];
#pragma unroll
    for (int j = 0; j < PJ; j += 2) jj[j / 2] = bp_pk2((float)j, (float)(j + 1));
    const unsigned long long mm = bp_pk2(kMagic, kMagic);

    for (int bt = 0; bt < nbt; ++bt) {
        const int st = bt & 1;
        const int cnt = min(kBatch, nq - bt * kBatch);
        // the next batch goes into the other half of the ring, which this warp
        // finished reading in the previous iteration
        if (bt + 1 < nbt)
            issue_batch(a, dys, sub, S, g, (bt + 1) * kBatch, min(kBatch, nq - (bt + 1) * kBatch), wl, X0, Y0,
                        xmax, ymax, my_win + (size_t)(st ^ 1) * kBatch * wl, my_slot + (st ^ 1) * kBatch,
                        &my_full[st ^ 1]);
        if (!mbar_wait(&my_full[st], (uint32_t)((bt >> 1) & 1), kWaitLimit)) {
            // a copy never landed: report, give the batch in flight a bounded
            // chance to land, and skip the rest (the block still meets at the
            // final barrier; the call returns the error)
            if (lane == 0) atomicExch(a.err, kErrTimeout);
            if (bt + 1 < nbt) mbar_wait(&my_full[st ^ 1], (uint32_t)(((bt + 1) >> 1) & 1), 1u << 16);
            break;
        }
        const float2* wb = my_win + (size_t)st * kBatch * wl;
        // the row's pair index is off + floor(beta) + floor(j sin + frac): two
        // magic-biased integers, so the base carries -2 kMagicBits
        const uint32_t wbase = smem_u32(wb) - ((uint32_t)kMagicBits << 4);
#pragma unroll
        for (int i = 0; i < kBatch; ++i) {
            if (i >= cnt) break;
            const float4 A = *reinterpret_cast<const float4*>(my_slot + st * kBatch + i);   // sin, sin, cos_h, cos_l
            const float4 B = *reinterpret_cast<const float4*>(&my_slot[st * kBatch + i].m); // m, 1 - m, f0, off
            const float b0 = fmaf(le, A.w, fmaf(le, A.z, B.z));      // beta - floor(beta_tile), this column
            const float tb = __fadd_rd(b0, kMagic);
            const float frac = __fsub_rn(b0, __fsub_rn(tb, kMagic));  // b0 - floor(b0), one rounding at most
            const uint32_t row = wbase + ((uint32_t)(__float_as_int(tb) + __float_as_int(B.w)) << 3);
            const float m = B.x, om = B.y;
            const unsigned long long sn2 = bp_pk2(A.x, A.y), fr2 = bp_pk2(frac, frac);
#ifdef MC_CHECKED
            const int wofs = (__float_as_int(tb) - kMagicBits) + __float_as_int(B.w) - i * wl;   // window offset
            const float sn = A.x;
#endif
#pragma unroll
            for (int j = 0; j < PJ; j += 2) {
                if (j >= pj) break;
                float dx, dy;
#ifdef MC_CHECKED
                float2 y0, y1;
                // the same arithmetic in C++, each pair index checked against
                // the angle's window (0 <= offset <= WL - 1)
                const float2 b2 = __ffma2_rn(make_float2((float)j, (float)(j + 1)), make_float2(sn, sn),
                                             make_float2(frac, frac));
                const float2 t2 = __fadd2_rd(b2, make_float2(kMagic, kMagic));
                const float2 fb2 = __fadd2_rn(t2, make_float2(-kMagic, -kMagic));
                dx = b2.x - fb2.x;
                dy = b2.y - fb2.y;
                const int o0 = wofs + (__float_as_int(t2.x) - kMagicBits);
                const int o1 = wofs + (__float_as_int(t2.y) - kMagicBits);
                const float2* win = wb + (size_t)i * wl;
                y0 = make_float2(0.0f, 0.0f);
                y1 = make_float2(0.0f, 0.0f);
                if (o0 >= 0 && o0 <= wl - 1) y0 = win[o0]; else atomicExch(a.err, kErrBounds);
                if (o1 >= 0 && o1 <= wl - 1) y1 = win[o1]; else atomicExch(a.err, kErrBounds);
#else
                float2 y0, y1;
                bp_two_rows(jj[j / 2], sn2, fr2, mm, row, dx, dy, y0, y1);
#endif
                acc[j] = fmaf(__saturatef(fmaf(-dx, m, 1.0f)), y0.x,
                              fmaf(__saturatef(fmaf(dx, m, om)), y0.y, acc[j]));
                acc[j + 1] = fmaf(__saturatef(fmaf(-dy, m, 1.0f)), y1.x,
                                  fmaf(__saturatef(fmaf(dy, m, om)), y1.y, acc[j + 1]));
            }
        }
        __syncwarp();
    }
    // fixed-order sum of the eight angle groups (reusing the window buffers
    // once every warp is done with them)
    __syncthreads();
    float* s_red = reinterpret_cast<float*>(s_win);                         // [kGroups][PJ][32]
#pragma unroll
    for (int j = 0; j < PJ; ++j) s_red[(g * PJ + j) * 32 + lane] = acc[j];
    __syncthreads();
    for (int j = g; j < pj; j += kGroups) {
        float v = 0.0f;
#pragma unroll
        for (int q = 0; q < kGroups; ++q) v += s_red[(q * PJ + j) * 32 + lane];
        const int r = r0 + j;
        if (c < n && r < n) a.out[(size_t)slot * n * n + (size_t)r * n + c] = v;
    }
}

// Residency: 4 blocks (32 warps) per SM at 64 registers for tiles of up to 16
// rows; 28-row tiles take 2 blocks per SM with up to 128 registers, and pay
// the per-angle set-up (slot constants, the column's beta, the window) once
// per 28 rows.
template <int PJ>
constexpr int bp_min_blocks() { return PJ > 16 ? 2 : 4; }

template <int PJ, bool SUB>
__global__ void __launch_bounds__(256, bp_min_blocks<PJ>()) k_backproject(BpArgs a)
{
    pdl_wait();
    pdl_trigger();
    bp_block<PJ, SUB>(a, blockIdx.x, blockIdx.y, blockIdx.z, PJ);
}

// Batched: the tiles of every slice of the launch (all angles, one slot),
// every slice with tile height PJ (the batch launches one such class per
// tile height).
template <int PJ>
__global__ void __launch_bounds__(256, bp_min_blocks<PJ>()) k_backproject_batch_pj(const BpArgs* __restrict__ args,
                                                                 const BatchBlock* __restrict__ map)
{
    pdl_wait();
    pdl_trigger();
    const BatchBlock m = map[blockIdx.x];
    const BpArgs& a = args[m.slice];
    const int tx = (a.n + 31) / 32;
    bp_block<PJ, false>(a, m.block % tx, m.block / tx, 0, PJ);
}

}  // namespace

int backproject_window(int pj) { return ((int)std::ceil(std::sqrt(31.0 * 31.0 + (pj - 1.0) * (pj - 1.0))) + 7) & ~1; }

size_t backproject_smem_bytes(int pj)
{
    const size_t win = (size_t)kGroups * kRing * kBatch * backproject_window(pj) * sizeof(float2);
    const size_t red = (size_t)kGroups * pj * 32 * sizeof(float);
    return 128 + kGroups * kRing * kBatch * sizeof(AngSlot) + std::max(win, red);
}

#define MC_BP_INSTANCES(X) \
    X(4, false) X(8, false) X(14, false) X(16, false) X(28, false) \
    X(4, true) X(8, true) X(14, true) X(16, true) X(28, true)

cudaError_t backproject_prepare()
{
    cudaError_t e = cudaSuccess;
#define MC_BP_ATTR(P, B)                                                                   \
    if (e == cudaSuccess)                                                                 \
        e = cudaFuncSetAttribute(k_backproject<P, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)backproject_smem_bytes(P));
    MC_BP_INSTANCES(MC_BP_ATTR)
#undef MC_BP_ATTR
#define MC_BPB_ATTR(P, B)                                                                 \
    if (e == cudaSuccess && !B)                                                           \
        e = cudaFuncSetAttribute(k_backproject_batch_pj<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)backproject_smem_bytes(P));
    MC_BP_INSTANCES(MC_BPB_ATTR)
#undef MC_BPB_ATTR
    return e;
}

int backproject_tiles(int n, int pj) { return ((n + 31) / 32) * ((n + pj - 1) / pj); }

cudaError_t launch_backproject_batch(const BpArgs* args, const BatchBlock* map, int nblocks, int pj,
                                     cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
#define MC_BPB_LAUNCH(P, B)                                                               \
    if (!B && pj == P)                                                                    \
        return pdl_launch(k_backproject_batch_pj<P>, dim3(nblocks), dim3(256), backproject_smem_bytes(P), s, \
                          args, map);
    MC_BP_INSTANCES(MC_BPB_LAUNCH)
#undef MC_BPB_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t launch_backproject(const BpArgs& a_in, cudaStream_t s)
{
    BpArgs a = a_in;
    a.wl = backproject_window(a.pj);
    if (a.wl > a.Pb) return cudaErrorInvalidValue;
    const dim3 grid((a.n + 31) / 32, (a.n + a.pj - 1) / a.pj, a.n_slots);
    const size_t smem = backproject_smem_bytes(a.pj);
    const bool sub = a.sel.subsets > 1;      // one angle subset per launch
#define MC_BP_LAUNCH(P, B)                                     \
    if (a.pj == P && sub == B) {                               \
        return pdl_launch(k_backproject<P, B>, grid, dim3(256), smem, s, a);   \
    }
    MC_BP_INSTANCES(MC_BP_LAUNCH)
#undef MC_BP_LAUNCH
    return cudaErrorInvalidValue;
}

}  // namespace mcg
