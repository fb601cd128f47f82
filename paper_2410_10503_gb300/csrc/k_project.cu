// K3 Joseph forward projection A w, ray-driven, with the dual update of
// Algorithm 1 step (ii) fused into its epilogue (arXiv 2410.10503, Sec. II-A
// and Algorithm 1: y_i^{k+1} = prox_{sigma f_i^*}(y_i^k + sigma A_i x^{k+1})).
//
// Rays are processed in warp-wide groups of up to 32 consecutive bins of one
// angle.  Work items are ranges of groups that share a driving axis, cut on
// the host so that every item has the same number of samples, and dealt to
// the consumer warps on the host (entry p of an item goes to warp p % W, slot
// p / W; an entry {-1, 0} is an empty slot); one block per
// SM takes `ipb` consecutive items and streams the whole warped image through
// shared memory for each, in chunks of LC lines.  One producer warp issues a
// bulk TMA copy (cp.async.bulk) per chunk into a ring of NS buffers (5; 3 for
// 16-line chunks and for 8-line chunks of large images); the consumer warps
// wait on the chunk's "full" mbarrier and release it through its "empty"
// mbarrier, so warps drift by up to NS - 1 chunks instead of meeting at a
// block barrier every chunk.  A block has W consumer warps (forward_warps: 15
// where 16-line chunks are sampled in two parts, whose state takes up to 128
// registers a thread; 23 at 80 registers for every other shape).
//
// A group visits only the chunks its rays cross.  A sample is an FMA for the
// position, one round-down add whose bits give both floor and shared address,
// one 8-byte shared load of the (w, next - w) pair and one FMA.  A ray's
// position is carried as an integer plus a float fraction: computed in
// float-pair arithmetic at its first line, advanced between chunks by the
// angle's exact integer/fraction split of LC * t, and stepped by j * t inside
// a chunk, so interpolation weights stay exact to ~1e-6 px.  A chunk is
// sampled in parts of CL lines (CL = LC, or 8 for a 16-line chunk on layouts
// with the narrow guard); every line has G = a.guard >= 2 CL + 1 zero pairs
// in front and at least G behind (P >= n + 2 G), and each part's starting
// pair index ui is clamped to [CL - 1, G + n + CL - 1].  With |t| <= 1 and a
// fraction in [0, 1] a part's samples lie at pair indices ui - (CL - 1) ..
// ui + CL, so every lane stays inside its line (at most index
// G + n + 2 CL - 1 <= P - 1); and a lane is clamped only when all of its
// samples in the part fall on zero pairs (indices up to 2 CL - 1 <= G - 2 in
// front, from G + n behind), where the clamped samples read zeros too.  So
// the rays of a group that leave the image inside a chunk, or miss it, need
// no predication and no separate edge path.
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase; false after `limit` failed polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try(addr, parity)) return true;
    return false;
}

// The producer's wait for a free stage: bounded, and it also gives up as soon
// as a consumer has raised the block's failure flag (the consumers that left
// will never release the stage).
__device__ __forceinline__ bool mbar_wait_or_flag(uint64_t* bar, uint32_t parity, uint32_t limit,
                                                  const int* flag)
{
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try(addr, parity)) return true;
        if ((it & 63u) == 63u && *(const volatile int*)flag) return false;
    }
    return false;
}

// Before the producer leaves: every copy it issued has landed, so no bulk
// copy is still writing into the block's shared memory when the block ends.
// Copies g in [issued - stages, issued) may still be in flight (older ones
// were waited for by the consumers before the producer could reuse their
// stage); each completes the phase g / stages of its stage's full barrier.
// Bounded: a copy that never lands leaves after `limit` polls with the error
// word already set.
__device__ __forceinline__ void drain_copies(uint64_t* full, int issued, int stages, uint32_t limit)
{
    for (int g = max(0, issued - stages); g < issued; ++g)
        mbar_wait(&full[g % stages], (uint32_t)((g / stages) & 1), limit);
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

// L2 prefetch of this block's share of a gate's CSR of D_i^T (row pointers
// and entries), as 16-byte-aligned bulk prefetches inside each array's range.
__device__ __forceinline__ void prefetch_span(const void* base, size_t bytes, int part, int parts)
{
    const uintptr_t b0 = (uintptr_t)base, b1 = b0 + bytes;
    uintptr_t s = b0 + bytes * part / parts, e = b0 + bytes * (part + 1) / parts;
    s = (s + 15) & ~(uintptr_t)15;
    e = min(e, b1) & ~(uintptr_t)15;
    if (e > s)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
}

__device__ __forceinline__ void prefetch_csr(const FwdArgs& a, int gate, int part, int parts)
{
    const size_t n2 = (size_t)a.n * a.n;
    const int* rp = a.pf_rowptr + (size_t)gate * (n2 + 1);
    prefetch_span(rp, (n2 + 1) * sizeof(int), part, parts);
    prefetch_span(a.pf_ent + a.pf_ent_off[gate], (size_t)__ldg(rp + n2) * sizeof(int2), part, parts);
}

constexpr uint32_t kWaitLimit = 1u << 24;   // polls before a stage wait gives up (unless the launch sets one)
constexpr int kMaxConsumers = 23;            // the most consumer warps of any instance (forward_warps)

#ifdef MC_CHECKED
// The samples of one ray over the LC lines of a chunk in C, the form used by
// MC_CHECKED builds: the magic constant of line j is kMagic + j * P; adding it
// with round-down leaves floor(w) + j * P in the low mantissa bits, so the
// pair's index is ibase + bits with ibase = ui - kMagicBits, and every pair
// index is checked against its line (0 <= ui + floor(w) <= P - 2); a failed
// check sets the error word and the sample reads zero.
__device__ __forceinline__ float2 load_pair(const float2* stage, int idx, int j, int P, int* err)
{
#ifdef MC_CHECKED
    const int q = idx - j * P;
    if (q < 0 || q > P - 2) {
        atomicExch(err, kErrBounds);
        return make_float2(0.0f, 0.0f);
    }
#endif
    return stage[idx];
}

template <int LC>
__device__ __forceinline__ float sample_lines(const float2* stage, int ibase, float fr, float t, const float* mj,
                                              float acc, int P, int* err)
{
#pragma unroll
    for (int j = 0; j < LC; j += 2) {
        const float2 w2 = __ffma2_rn(make_float2(-(float)j, -(float)(j + 1)), make_float2(t, t),
                                     make_float2(fr, fr));
        const float2 t2 = __fadd2_rd(w2, make_float2(mj[j], mj[j + 1]));
        const float2 d2 = __fadd2_rn(t2, make_float2(-mj[j], -mj[j + 1]));     // floor(w), exact
        const float2 f2 = __ffma2_rn(d2, make_float2(-1.0f, -1.0f), w2);       // w - floor(w), exact
        const float2 v0 = load_pair(stage, ibase + __float_as_int(t2.x), j, P, err);
        acc += fmaf(f2.x, v0.y, v0.x);
        const float2 v1 = load_pair(stage, ibase + __float_as_int(t2.y), j + 1, P, err);
        acc += fmaf(f2.y, v1.y, v1.x);
    }
    return acc;
}
#endif

// Two FP32 values as one 64-bit register pair (the operand form of the
// f32x2 instructions).
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

// The same samples written as PTX on packed pairs:
// the line constants jj = (-j, -(j+1)) and mm = (magic_j, magic_{j+1}) stay
// in registers for the whole kernel, tt = (t, t) and ff = (fr, fr) are
// packed once per group and chunk, and gbase = shared address of the stage
// + 8 (ui - kMagicBits), so a sample's address is one multiply-add of its
// round-down bits.  Same arithmetic, bit for bit, as sample_lines.
template <int LC>
__device__ __forceinline__ float sample_interior(uint32_t gbase, unsigned long long tt, unsigned long long ff,
                                                 const unsigned long long* jj, const unsigned long long* mm,
                                                 float acc)
{
#pragma unroll
    for (int q = 0; q < LC / 2; ++q) {
        float f0, f1, v0x, v0y, v1x, v1y;
        asm volatile(
            "{\n\t"
            ".reg .b64 w2, t2, d2, f2;\n\t"
            ".reg .b32 b0, b1, a0, a1;\n\t"
            "fma.rn.f32x2 w2, %6, %7, %8;\n\t"
            "add.rm.f32x2 t2, w2, %9;\n\t"
            "sub.rn.f32x2 d2, t2, %9;\n\t"
            "sub.rn.f32x2 f2, w2, d2;\n\t"
            "mov.b64 {b0, b1}, t2;\n\t"
            "mov.b64 {%0, %1}, f2;\n\t"
            "mad.lo.u32 a0, b0, 8, %10;\n\t"
            "mad.lo.u32 a1, b1, 8, %10;\n\t"
            "ld.shared.v2.f32 {%2, %3}, [a0];\n\t"
            "ld.shared.v2.f32 {%4, %5}, [a1];\n\t"
            "}"
            : "=f"(f0), "=f"(f1), "=f"(v0x), "=f"(v0y), "=f"(v1x), "=f"(v1y)
            : "l"(jj[q]), "l"(tt), "l"(ff), "l"(mm[q]), "r"(gbase));
        acc += fmaf(f0, v0y, v0x);
        acc += fmaf(f1, v1y, v1x);
    }
    return acc;
}

// Per-warp, per-slot constants of the chunk loop, in shared memory: the
// slope twice (one 16-byte load gives the packed operand of the position
// FMA) and the exact split of the per-chunk advance.
struct SlotState {
    float t0, t1, step_frac;
    int step_int;
};

// A slot's group {angle, first bin} and the angle's Joseph table, fetched by
// one lane per slot at the start of an item so that the slots' dependent
// global loads are in flight together.
struct SlotRec {
    FwdAngle T;
    int2 grp;
};

// BANDED (angle-subset launches): an item also names a band of chunks
// [band * cpb, (band + 1) * cpb); its rays' partial sums over that band go to
// a.part[band] and k_forward_combine adds the bands in order and runs the
// epilogue.  Items then hold several times more ray groups and stream only
// their band of the image, where an unbanded subset item would stream the
// whole image for a few groups.
// One block's work: items bx * ipb .. of the launch's item table for gate
// slot `slot`; nbx = blocks sharing the table (the CSR prefetch is split
// among them).
template <int RPT, int LC, int NS, int CL, int W, bool BANDED>
__device__ __forceinline__ void forward_block(const FwdArgs& a, int bx, int slot, int nbx, SlotState* s_slot,
                                              SlotRec* s_rec)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxStages;
    int* s_flag = reinterpret_cast<int*>(smem + 96);
    float2* stage0 = reinterpret_cast<float2*>(smem + 128);
    const size_t stage_pairs = (size_t)LC * a.P;   // one chunk: LC whole lines

    const int n = a.n, nb = a.nb;
    const int nch = layout_lines(n) / LC;        // the layouts hold whole chunks (zero lines past n)
    // this launch's item table: all angles, or the drawn block's angle subset
    const int sub = sel_subset(a.sel, slot);
    const RayItem* items = a.sub_off ? a.items + a.sub_off[sub] : a.items;
    const int n_items = a.sub_off ? a.sub_off[sub + 1] - a.sub_off[sub] : a.n_items;
    const int it0 = bx * a.ipb;
    const int n_it = min(a.ipb, n_items - it0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], W);
        }
        *s_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t wlim = a.wait_limit ? a.wait_limit : kWaitLimit;

    // ---- producer warp: fill the ring, item after item ----------------------
    // On a failure (its own wait for a free stage ran out, or a consumer raised
    // the block's flag) the producer issues nothing more and waits for the
    // copies it has in flight before it leaves.
    if (warp == W) {
        if (a.stall) return;          // test of the waits' failure path: no copies in flight
        if (lane == 0) {
            int issued = 0;           // copies issued so far (ring position of the next one)
            if constexpr (BANDED) {
                // running chunk count q over the items' bands
                bool stop = false;
                for (int it = 0; it < n_it && !stop; ++it) {
                    const RayItem item = items[it0 + it];
                    const float2* src = (item.dir ? a.lcol : a.lrow) + slot * a.layout_stride;
                    const int cb0 = item.band * a.cpb, cb1 = min(nch, cb0 + a.cpb);
                    for (int c = cb0; c < cb1; ++c) {
                        const int q = issued;
                        const int st = q % NS;
                        if (q >= NS &&
                            !mbar_wait_or_flag(&empty[st], (uint32_t)((q / NS - 1) & 1), wlim, s_flag)) {
                            atomicExch(s_flag, 1);
                            atomicExch(a.err, kErrTimeout);
                            stop = true;
                            break;
                        }
                        if (*(volatile int*)s_flag) { stop = true; break; }
                        bulk_load(stage0 + st * stage_pairs, src + (size_t)c * stage_pairs,
                                  (uint32_t)(stage_pairs * sizeof(float2)), &full[st]);
                        ++issued;
                    }
                }
            } else {
                for (int g = 0; g < n_it * nch; ++g) {
                    const int it = g / nch, c = g - it * nch;
                    const float2* src = (items[it0 + it].dir ? a.lcol : a.lrow) + slot * a.layout_stride;
                    const int st = g % NS;
                    if (g >= NS &&
                        !mbar_wait_or_flag(&empty[st], (uint32_t)((g / NS - 1) & 1), wlim, s_flag)) {
                        atomicExch(s_flag, 1);
                        atomicExch(a.err, kErrTimeout);
                        break;
                    }
                    if (*(volatile int*)s_flag) break;
                    bulk_load(stage0 + st * stage_pairs, src + (size_t)c * stage_pairs,
                              (uint32_t)(stage_pairs * sizeof(float2)), &full[st]);
                    ++issued;
                }
            }
            drain_copies(full, issued, NS, wlim);
        }
        // off the ring's critical path: prefetch the CSR the iteration's
        // transpose warp will read (a.pf_rowptr is set for one-slot SPDHG launches)
        if (lane == 1 && a.pf_rowptr && a.n_slots == 1) prefetch_csr(a, sel_gate(a.sel, slot), bx, nbx);
        return;
    }

    // ---- consumers ------------------------------------------------------------
    const int gate = sel_gate(a.sel, slot);
    const float h = 0.5f * (float)(n - 1);
    const float hb = 0.5f * (float)(nb - 1);
    const int guard = a.guard;
    const float off = h + (float)guard;
    static_assert(LC % CL == 0, "a chunk is whole sampling parts");
    float mj[CL];
#pragma unroll
    for (int j = 0; j < CL; ++j) mj[j] = kMagic + (float)(j * a.P);
    SlotState* my = s_slot + warp * RPT;
    unsigned long long jj[CL / 2], mm[CL / 2];
#pragma unroll
    for (int q = 0; q < CL / 2; ++q) {
        jj[q] = pk2(-(float)(2 * q), -(float)(2 * q + 1));
        mm[q] = pk2(mj[2 * q], mj[2 * q + 1]);
    }
    // clamp of a part's first-line pair index (see the file comment; a chunk is
    // sampled in LC / CL parts of CL lines, each clamped on its own)
    const int ui_lo = CL - 1, ui_hi = guard + n + CL - 1;

    int q_run = 0;                        // BANDED: chunks consumed so far
    for (int it = 0; it < n_it; ++it) {
        const RayItem item = items[it0 + it];
        const int cb0 = BANDED ? item.band * a.cpb : 0;
        const int cb1 = BANDED ? min(nch, cb0 + a.cpb) : nch;
        // this warp's groups: item.begin + warp + m * W
        const int ns = max(0, min(RPT, (item.end - item.begin - warp + W - 1) / W));
        float frac[RPT], acc[RPT];
        int ui[RPT];
        int my_lo = nch, my_hi = -1;      // lane m < RPT: chunk range of slot m
        SlotRec* rec = s_rec + warp * RPT;
        if (lane < ns) {
            SlotRec r;
            r.grp = __ldg(a.groups + item.begin + warp + lane * W);
            if (r.grp.x >= 0) r.T = a.ang[r.grp.x];
            rec[lane] = r;
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            acc[m] = 0.0f; frac[m] = 0.0f; ui[m] = 0;
            if (m >= ns) continue;
            const int2 grp = rec[m].grp;
            if (grp.x < 0) continue;                            // empty slot of the item's deal
            const int b = min(grp.y + lane, nb - 1);           // idle lanes repeat the last ray
            const FwdAngle T = rec[m].T;
            const float B = (float)b - hb;                      // exact
            const float t = T.t_hi;
            // lines with a non-zero weight have u in (guard - 1, guard + n);
            // widen by up to two lines (extra samples read zeros)
            const float u0 = fmaf(h, t, fmaf(B, T.inv_hi, off));
            int lo = n, hi = -1;
            if (fabsf(t) < 1e-6f) {
                if (u0 > (float)guard - 2.0f && u0 < (float)(guard + n) + 1.0f) { lo = 0; hi = n - 1; }
            } else {
                const float e1 = (u0 - (float)(guard + n)) / t;
                const float e3 = (u0 - (float)(guard - 1)) / t;
                const float l_lo = fmaxf(floorf(fminf(e1, e3)) - 1.0f, 0.0f);
                const float l_hi = fminf(ceilf(fmaxf(e1, e3)) + 1.0f, (float)(n - 1));
                if (l_lo <= l_hi) { lo = (int)l_lo; hi = (int)l_hi; }
            }
            // chunks of the group: the union of its rays' ranges
            const int lo_min = __reduce_min_sync(0xffffffffu, lo);
            const int hi_max = __reduce_max_sync(0xffffffffu, hi);
            const int c_lo = (hi_max >= lo_min) ? (BANDED ? max(lo_min / LC, cb0) : lo_min / LC) : nch;
            const int c_hi = (hi_max >= lo_min) ? (BANDED ? min(hi_max / LC, cb1 - 1) : hi_max / LC) : -1;
            if (lane == m) { my_lo = c_lo; my_hi = c_hi; }
            if (lane == 0) my[m] = SlotState{t, t, T.step_frac, T.step_int};
            // position at the group's first line L = c_lo * LC:
            // u(L) = B inv - (L - h) t + h + guard, in float pairs
            const float L = (float)(min(c_lo, nch - 1) * LC) - h;   // exact
            float ph, pl, qh, ql, s, e, s2, e2;
            mul_df(B, T.inv_hi, T.inv_lo, ph, pl);
            mul_df(-L, T.t_hi, T.t_lo, qh, ql);
            two_sum(ph, qh, s, e);
            two_sum(s, off, s2, e2);
            split_int_frac(s2, (pl + ql) + (e + e2), ui[m], frac[m]);
        }
        __syncwarp();

        for (int ch = cb0; ch < cb1; ++ch) {
            const int g = BANDED ? q_run++ : it * nch + ch;
            const int st = g % NS;
            // one verdict per warp, so that all lanes leave or none does
            if (!__all_sync(0xffffffffu, mbar_wait_or_flag(&full[st], (uint32_t)((g / NS) & 1), wlim, s_flag))) {
                // this wait ran out, or another warp's did: the producer sees
                // the flag, stops issuing and drains the copies it has in
                // flight before the block ends
                atomicExch(s_flag, 1);
                atomicExch(a.err, kErrTimeout);
                return;
            }
            const float2* sp = stage0 + st * stage_pairs;
            // slots whose group crosses this chunk, one bit each
            const uint32_t act = __ballot_sync(0xffffffffu, ch >= my_lo && ch <= my_hi);
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (!((act >> m) & 1u)) continue;
                const float4 gs = *reinterpret_cast<const float4*>(my + m);   // {t, t, step_frac, step_int}
#pragma unroll
                for (int part = 0; part < LC / CL; ++part) {
                    const int ib = min(max(ui[m], ui_lo), ui_hi) - kMagicBits;
                    const float2* pp = sp + (size_t)part * CL * a.P;
#ifdef MC_CHECKED
                    acc[m] = sample_lines<CL>(pp, ib, frac[m], gs.x, mj, acc[m], a.P, a.err);
#else
                    const uint32_t gbase = (uint32_t)__cvta_generic_to_shared(pp) + ((uint32_t)ib << 3);
                    acc[m] = sample_interior<CL>(gbase, pk2(gs.x, gs.y), pk2(frac[m], frac[m]), jj, mm, acc[m]);
#endif
                    // advance to the first line of the next part: u -= CL * t
                    float nf = frac[m] - gs.z;
                    int nu = ui[m] - __float_as_int(gs.w);
                    if (nf < 0.0f) { nf += 1.0f; nu -= 1; }
                    frac[m] = nf;
                    ui[m] = nu;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }

        // ---- epilogue ---------------------------------------------------------
        // slots' groups and angle steps come from the staged records; every
        // slot's y and d are loaded before any store, so their latencies overlap
        if constexpr (BANDED) {
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (m >= ns) break;
                const int2 grp = rec[m].grp;
                const int b = grp.y + lane;
                if (grp.x >= 0 && b < nb) a.part[((size_t)item.band * a.na + grp.x) * nb + b] = acc[m];
            }
        } else {
            float yo[RPT], dv[RPT];
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                yo[m] = 0.0f; dv[m] = 0.0f;
                if (m >= ns || a.mode == 0) continue;
                const int2 grp = rec[m].grp;
                const int b = grp.y + lane;
                if (grp.x < 0 || b >= nb) continue;
                const size_t gi = ((size_t)gate * a.na + grp.x) * nb + b;
                if (a.store == 0) {
                    yo[m] = a.y[gi];
                    dv[m] = a.d[gi];
                } else {
                    yo[m] = load_store(a.yh[gi], a.store);
                    dv[m] = load_store(a.dh[gi], a.store);
                }
            }
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                if (m >= ns) break;
                const int2 grp = rec[m].grp;
                const int k = grp.x, b = grp.y + lane;
                if (k < 0 || b >= nb) continue;
                const float delta = rec[m].T.delta;
                const float val = delta * acc[m];
                const size_t idx = (size_t)k * nb + b;
                if (a.mode == 0) {
                    a.out[(size_t)slot * a.na * nb + idx] = val;
                } else {
                    const size_t gi = (size_t)gate * a.na * nb + idx;
                    float yn;
                    if (a.store == 0) {
                        yn = (yo[m] + a.sigma * (val - dv[m])) * a.inv_den;
                        a.y[gi] = yn;
                    } else {
                        // reduced-precision d and y: arithmetic in float32, the new
                        // y rounded on store and the increment taken from stored values
                        const float yf = (yo[m] + a.sigma * (val - dv[m])) * a.inv_den;
                        const unsigned short q = to_store(yf, a.store);
                        a.yh[gi] = q;
                        yn = load_store(q, a.store);
                    }
                    // dy pairs scaled by the angle's step: (m dy[b], m dy[b+1])
                    const float v = delta * (yn - yo[m]);
                    float* dyp = reinterpret_cast<float*>(a.dy + slot * a.dy_stride + (size_t)k * a.Pb + a.Gb + b);
                    dyp[0] = v;
                    dyp[-1] = v;
                }
            }
        }
        __syncwarp();
    }
}

template <int RPT, int LC, int NS, int CL, bool BANDED, int W = forward_warps(LC, CL)>
__global__ void __launch_bounds__(32 * (W + 1), 1) k_forward(FwdArgs a)
{
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) SlotState s_slot[W * RPT];
    __shared__ __align__(16) SlotRec s_rec[W * RPT];
    forward_block<RPT, LC, NS, CL, W, BANDED>(a, blockIdx.x, blockIdx.y, gridDim.x, s_slot, s_rec);
}

// Batched: the blocks of every slice of the launch, each on its slice's item
// table with its slice's arguments (all angles, one slot, no bands); every
// slice of the launch has LC lines per chunk and an NS-stage ring (the batch
// launches one such class per chunk size and ring).
template <int RPT, int LC, int NS, int CL, int W = forward_warps(LC, CL)>
__global__ void __launch_bounds__(32 * (W + 1), 1) k_forward_batch_lc(const FwdArgs* __restrict__ args,
                                                                const BatchBlock* __restrict__ map)
{
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) SlotState s_slot[W * RPT];
    __shared__ __align__(16) SlotRec s_rec[W * RPT];
    const BatchBlock m = map[blockIdx.x];
    forward_block<RPT, LC, NS, CL, W, false>(args[m.slice], m.block, 0, m.nblocks, s_slot, s_rec);
}

// Sum of the bands' partial ray sums in band order, then the epilogue of
// k_forward (store, or the dual update of Algorithm 1 (ii)); one thread per
// ray of the launch's angle subset.
__global__ void __launch_bounds__(256) k_forward_combine(FwdArgs a)
{
    pdl_wait();
    pdl_trigger();
    const int slot = blockIdx.y;
    const int nb = a.nb;
    const int S = a.sel.subsets > 1 ? a.sel.subsets : 1;
    const int sub = sel_subset(a.sel, slot);
    const int na_s = (a.na - sub + S - 1) / S;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= na_s * nb) return;
    const int m = idx / nb, b = idx - m * nb;
    const int k = sub + m * S;
    float accv = 0.0f;
    for (int band = 0; band < a.nbands; ++band) accv += a.part[((size_t)band * a.na + k) * nb + b];
    const float delta = __ldg(&a.ang[k].delta);
    const float val = delta * accv;
    const size_t ki = (size_t)k * nb + b;
    if (a.mode == 0) {
        a.out[(size_t)slot * a.na * nb + ki] = val;
        return;
    }
    const int gate = sel_gate(a.sel, slot);
    const size_t gi = (size_t)gate * a.na * nb + ki;
    float yo, yn;
    if (a.store == 0) {
        yo = a.y[gi];
        yn = (yo + a.sigma * (val - a.d[gi])) * a.inv_den;
        a.y[gi] = yn;
    } else {
        yo = load_store(a.yh[gi], a.store);
        const float yf = (yo + a.sigma * (val - load_store(a.dh[gi], a.store))) * a.inv_den;
        const unsigned short q = to_store(yf, a.store);
        a.yh[gi] = q;
        yn = load_store(q, a.store);
    }
    const float v = delta * (yn - yo);
    float* dyp = reinterpret_cast<float*>(a.dy + slot * a.dy_stride + (size_t)k * a.Pb + a.Gb + b);
    dyp[0] = v;
    dyp[-1] = v;
}

}  // namespace

int forward_groups_per_block(int rpt, int warps) { return warps * rpt; }



// static shared memory of the largest instance: the slot tables plus room for
// the alignment padding the compiler may place between them
int forward_static_smem() { return (int)(kMaxConsumers * 8 * (sizeof(SlotState) + sizeof(SlotRec))) + 256; }

size_t forward_smem_bytes(int lc, int P)
{
    return 128 + (size_t)forward_ring(lc, P) * lc * P * sizeof(float2);
}

// (group slots per warp, lines per chunk, ring stages, lines per clamped part)
#define MC_FWD_INSTANCES(X) \
    X(2, 2, 5, 2) X(4, 2, 5, 2) X(8, 2, 5, 2) X(2, 4, 5, 4) X(4, 4, 5, 4) X(8, 4, 5, 4) \
    X(2, 8, 5, 8) X(4, 8, 5, 8) X(8, 8, 5, 8) X(2, 8, 3, 8) X(4, 8, 3, 8) X(8, 8, 3, 8) \
    X(2, 16, 3, 16) X(4, 16, 3, 16) X(8, 16, 3, 16) X(2, 16, 3, 8) X(4, 16, 3, 8) X(8, 16, 3, 8)

cudaError_t forward_prepare(int max_smem)
{
    cudaError_t e = cudaSuccess;
#define MC_SET_ATTR(R, L, NS, CL)                                                                  \
    if (e == cudaSuccess)                                                                         \
        e = cudaFuncSetAttribute(k_forward<R, L, NS, CL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 max_smem);                                                       \
    if (e == cudaSuccess)                                                                         \
        e = cudaFuncSetAttribute(k_forward<R, L, NS, CL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 max_smem);                                                       \

    MC_FWD_INSTANCES(MC_SET_ATTR)
#undef MC_SET_ATTR
#define MC_SET_ATTR_B(R, L, NS, CL)                                                                \
    if (e == cudaSuccess)                                                                         \
        e = cudaFuncSetAttribute(k_forward_batch_lc<R, L, NS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 max_smem);
    MC_FWD_INSTANCES(MC_SET_ATTR_B)
#undef MC_SET_ATTR_B
    return e;
}

cudaError_t launch_forward(const FwdArgs& a_in, cudaStream_t s)
{
    FwdArgs a = a_in;
    a.stages = forward_ring(a.lc, a.P);
    a.cl = forward_part_lines(a.lc, a.guard);
    if (!forward_lines_fit(a.n, a.P, a.guard, a.lc) || a.P < a.n + 2 * a.guard) return cudaErrorInvalidValue;
    if (a.nbands > 1 && (a.n_slots != 1 || !a.part)) return cudaErrorInvalidValue;   // one partial buffer
    const dim3 grid((a.n_items + a.ipb - 1) / a.ipb, a.n_slots);
    const size_t smem = forward_smem_bytes(a.lc, a.P);
#define MC_LAUNCH(R, L, NS, CL)                                                           \
    if (a.rpt == R && a.lc == L && a.stages == NS && a.cl == CL) {                        \
        if (a.nbands > 1) {                                                               \
            cudaError_t e = pdl_launch(k_forward<R, L, NS, CL, true>, grid, dim3(32 * (forward_warps(L, CL) + 1)), \
                                       smem, s, a);                                        \
            if (e != cudaSuccess) return e;                                               \
            const int S = a.sel.subsets > 1 ? a.sel.subsets : 1;                          \
            const int rays = ((a.na + S - 1) / S) * a.nb;                                 \
            return pdl_launch(k_forward_combine, dim3((rays + 255) / 256, a.n_slots), dim3(256), 0, s, a); \
        } else {                                                                          \
            return pdl_launch(k_forward<R, L, NS, CL, false>, grid, dim3(32 * (forward_warps(L, CL) + 1)), \
                              smem, s, a);                                                 \
        }                                                                                 \
    }
    MC_FWD_INSTANCES(MC_LAUNCH)
#undef MC_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t launch_forward_batch(const FwdArgs* args, const BatchBlock* map, int nblocks, int rpt,
                                 size_t smem_bytes, int lc, int stages, int cl, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    const size_t smem = smem_bytes;
#define MC_LAUNCH_B(R, L, NS, CL)                                                           \
    if (rpt == R && lc == L && stages == NS && cl == CL)                                    \
        return pdl_launch(k_forward_batch_lc<R, L, NS, CL>, dim3(nblocks), dim3(32 * (forward_warps(L, CL) + 1)), \
                          smem, s, args, map);
    MC_FWD_INSTANCES(MC_LAUNCH_B)
#undef MC_LAUNCH_B
    return cudaErrorInvalidValue;
}

}  // namespace mcg
