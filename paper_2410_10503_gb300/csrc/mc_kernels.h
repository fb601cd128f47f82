// Host-side launchers of the libmc kernels (one translation unit each).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mc_device.cuh"

namespace mcg {

// Which block a gate slot works on: list[slot] if list, else fixed if >= 0,
// else the slot index itself (PDHG: slot i is gate i).  With subsets = S > 1
// the value is a block j of the gate x angle-subset split: gate j / S, angle
// subset j % S (angles k = j % S + m S); subsets <= 1 means plain gates.
struct GateSel {
    const int* list;
    int fixed;
    int subsets;
    const int* pos;            // non-null (batched runs): {iteration within the epoch,
                               // epoch parity}; the entry is list[pos[1] * stride + pos[0]]
    int stride;
};

__device__ __forceinline__ int sel_block(const GateSel& s, int slot)
{
    return s.list ? s.list[s.pos ? s.pos[1] * s.stride + s.pos[0] : slot] : (s.fixed >= 0 ? s.fixed : slot);
}

// Batched launches over many independent slices (one context each): block b
// of the launch works on block `block` (of `nblocks`) of slice `slice`, with
// that slice's arguments args[slice].
struct BatchBlock {
    int slice, block, nblocks, pad;
};

// The gate sequence of one slice in batched iterations.  state holds, for each
// parity t of the iteration index, {iteration within the epoch, epoch parity};
// gates holds two epochs' gates (stride apart, by epoch parity).  The last
// kernel of an iteration of parity t writes state[t ^ 1] (the next iteration)
// and, when that starts an epoch, draws its n_blocks gates into the other half
// exactly as the one-slice draw does (Philox counter kctr, advanced by
// n_blocks); the kernels of the iteration read only state[t] and the current
// half, so nothing they read changes under them.
struct BatchDraw {
    uint64_t seed;
    uint32_t stream;
    int n_blocks;
    unsigned long long* kctr;
    const unsigned long long* thr;
    int* gates;
    int* state;                // [2][2]
    int stride;
};

__device__ __forceinline__ int sel_gate(const GateSel& s, int slot)
{
    const int v = sel_block(s, slot);
    return s.subsets > 1 ? v / s.subsets : v;
}

__device__ __forceinline__ int sel_subset(const GateSel& s, int slot)
{
    return s.subsets > 1 ? sel_block(s, slot) % s.subsets : 0;
}

// ---- K1: warp w = D_i x into the two line layouts (or a plain image) ------
struct WarpArgs {
    const float* x;            // n*n input image (shared by all slots)
    int n;
    const RigidGate* rigid;    // per gate, or null
    const float* field;        // per gate 2*n*n, or null
    int identity;              // 1: w = x (no motion; the ray transform alone)
    GateSel sel;
    int n_slots;
    float2* lrow;              // pair line layouts, slot stride layout_stride pairs
    float2* lcol;
    size_t layout_stride;
    int P;                     // line pitch (pairs)
    int guard;                 // zero pairs before each line's data (layout_guard)
    float* out;                // plain mode: n*n per slot
};
cudaError_t launch_warp_layouts(const WarpArgs& a, cudaStream_t s);
// batched: block b computes tile map[b].block of slice map[b].slice (one slot)
cudaError_t launch_warp_layouts_batch(const WarpArgs* args, const BatchBlock* map, int nblocks, cudaStream_t s);
int warp_layout_tiles(int n);
cudaError_t launch_warp_plain(const WarpArgs& a, cudaStream_t s);

// ---- K2: per-gate CSR of D_i^T --------------------------------------------
cudaError_t launch_csr_count(int n, const RigidGate* rg, const float* field, int* cnt,
                             cudaStream_t s);
cudaError_t launch_exclusive_scan(const int* in, int* out_rowptr, int len, int* scratch,
                                  int scratch_len, cudaStream_t s);
int scan_scratch_len(int len);
cudaError_t launch_csr_fill(int n, const RigidGate* rg, const float* field,
                            const int* rowptr, int* cursor, int2* ent, cudaStream_t s);
cudaError_t launch_csr_sort(int n, const int* rowptr, int2* ent, cudaStream_t s);

// ---- field VJP: out0/out1 = g * d(D_u x)/du_x, d(D_u x)/du_y (one gate) -----
cudaError_t launch_field_vjp(int n, const float* field, const float* x, const float* g,
                             float* out0, float* out1, cudaStream_t s);

// ---- K5 (+K7): v = sum_slots D_gate^T b_slot, then store or update ----------
struct WarpAdjArgs {
    int n;
    const int* rowptr;         // gate g: rowptr + g*(n*n+1)
    const int2* ent;           // gate g: ent + ent_off[g]
    const long long* ent_off;
    GateSel sel;
    int n_slots;
    const float* b;            // slot stride n*n
    // store mode
    float* out;
    // update mode (fused z / zbar / primal prox of Algorithm 1)
    float* z;
    const float* x_in;
    float* x_out;
    float coef;                // theta / p_i (uniform sampling)
    const float* coef_tab;     // non-null: theta / p_i per gate, read for the slot's block
    float tau;
    float prox_scale;          // 1 / (1 + 2 tau alpha)
    // non-null (a batched run with one slice in flight, the one-slice kernel):
    // the first warp of block 0 advances that slice's gate sequence from
    // iteration parity draw_t, as the batched kernel's first block does
    const BatchDraw* draw;
    int draw_t;
};
cudaError_t launch_warp_adjoint_store(const WarpAdjArgs& a, cudaStream_t s);
cudaError_t launch_warp_adjoint_update(const WarpAdjArgs& a, cudaStream_t s);
// the transpose warp and update of every slice in flight; the first block of
// each slice also advances that slice's gate sequence (draw[slice], parity t)
cudaError_t launch_warp_adjoint_update_batch(const WarpAdjArgs* args, const BatchBlock* map, int nblocks,
                                             const BatchDraw* draw, int t, cudaStream_t s);
int warp_adjoint_blocks(int n);

// ---- K3 (+K6): Joseph forward projection ------------------------------------
struct FwdArgs {
    const float2* lrow;
    const float2* lcol;
    size_t layout_stride;
    int P;
    const FwdAngle* ang;
    const int2* groups;        // ray groups {angle k, first bin}, rows-driven first
    const RayItem* items;      // group ranges
    int n_items;               // items (the largest subset's count when sub_off is set)
    const int* sub_off;        // angle-subset tables: items of subset s are
                               // items[sub_off[s] .. sub_off[s+1]), or null
    int nbands;                // > 1: items carry a band of cpb chunks; partial ray
    int cpb;                   //      sums go to part [nbands][na][nb] and a combine
    float* part;               //      kernel adds them and runs the epilogue
    int ipb;                   // items per block (one block per SM)
    int rpt;                   // group slots per consumer warp (2, 4, 8)
    int guard;                 // zero pairs before each line's data (>= 2 cl + 1)
    int lc;                    // lines per staged chunk (2, 4, 8, 16)
    int cl;                    // lines per sampled part of a chunk: forward_part_lines(lc, guard)
                               // (launch_forward sets it; batched argument tables carry it)
    int stages;                // ring stages: forward_ring(lc, P) (launch_forward sets it;
                               // batched argument tables carry it)
    int n, na, nb;
    GateSel sel;
    int n_slots;
    int mode;                  // 0: store A w; 1: dual update of Algorithm 1 (ii)
    float* out;                // mode 0: slot stride na*nb
    const float* d;            // mode 1: gate stride na*nb
    float* y;
    float2* dy;                // pairs, slot stride dy_stride, pitch Pb, guard Gb
    size_t dy_stride;
    int Pb, Gb;
    float sigma;
    float inv_den;             // 1 / (1 + sigma N / 2)
    int store;                 // mode 1: 0 d, y as float; 1 binary16; 2 bfloat16 (dh, yh)
    const unsigned short* dh;  // mode 1, store != 0: data and dual, gate stride na*nb
    unsigned short* yh;
    int* err;
    // optional (one slot): the CSR of D_i^T of the slot's gate (layout as in
    // WarpAdjArgs) is prefetched into L2 by an idle lane of each block's
    // producer warp, for the transpose warp at the end of the same iteration
    const int* pf_rowptr;
    const int2* pf_ent;
    const long long* pf_ent_off;
    unsigned wait_limit;       // polls before a ring wait gives up (0: the default 2^24)
    int stall;                 // 1: the producer issues no copies (tests the waits' failure path)
};
cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s);
// batched (all angles, one slot per slice, no bands): block b runs block
// map[b].block of slice map[b].slice's item table with that slice's lines per
// chunk (args[slice].lc: 16, 8, 4 or 2) and ring stages (args[slice].stages,
// forward_ring); every slice of the launch has lc lines per chunk sampled in
// parts of cl lines, a ring of `stages` stages (the kernel is compiled for
// these) and at most rpt group slots per warp; smem_bytes = the largest
// forward_smem_bytes of its slices
cudaError_t launch_forward_batch(const FwdArgs* args, const BatchBlock* map, int nblocks, int rpt,
                                 size_t smem_bytes, int lc, int stages, int cl, cudaStream_t s);
int forward_groups_per_block(int rpt, int warps);   // group slots of an item: warps x rpt
int forward_static_smem();           // static shared memory of the largest instance
size_t forward_smem_bytes(int lc, int P);
cudaError_t forward_prepare(int max_smem);

// ---- K4: pixel-driven gather backprojection ---------------------------------
struct BpArgs {
    GateSel sel;               // only the angle subset is used (all angles if subsets <= 1)
    const float2* dy;          // pairs, slot stride dy_stride, pitch Pb, guard Gb
    size_t dy_stride;
    int Pb, Gb;
    const BpAngle* ang;
    int n, na, nb;
    int n_slots;
    int pj;                    // pixels per thread along a column (4, 8, 14 or 16)
    float* out;                // slot stride n*n
    int* err;
    int wl;                    // staged window length (pairs), set by the launcher
};
cudaError_t launch_backproject(const BpArgs& a, cudaStream_t s);
// batched (all angles, one slot per slice): block b works on tile
// map[b].block of slice map[b].slice; every slice of the launch has tile
// height pj (args[slice].pj: 4, 8, 14, 16 or 28; a kernel compiled for it)
// and its own window length (args[slice].wl)
cudaError_t launch_backproject_batch(const BpArgs* args, const BatchBlock* map, int nblocks, int pj,
                                     cudaStream_t s);
int backproject_tiles(int n, int pj);
int backproject_window(int pj);
cudaError_t backproject_prepare();

// ---- misc -------------------------------------------------------------------
// thr: null for uniform sampling, else N cumulative thresholds (see k_draw_gates)
cudaError_t launch_draw_gates(uint64_t seed, uint32_t stream, unsigned long long* kctr,
                              uint64_t k0, int count, int n_gates, const unsigned long long* thr, int* out,
                              cudaStream_t s);
// write a na x nb sinogram into the padded, m_k-scaled pair layout of dy
// (guards stay zero)
cudaError_t launch_pad_sino(const float* y, float2* dy, const BpAngle* ang, int na, int nb,
                            int Pb, int Gb, cudaStream_t s);
// FP64 reductions, deterministic; result in out[0] (device)
enum { kRedSumSq = 0, kRedDiffSq = 1, kRedDot = 2 };
int reduce_parts();
cudaError_t launch_reduce(const float* a, const float* b, size_t len, int mode,
                          double* partial, double* out, cudaStream_t s);
// out[i] = a * x[i] + b * y[i]  (y may be null -> b ignored)
cudaError_t launch_axpby(float a, const float* x, float b, const float* y, float* out,
                         size_t len, cudaStream_t s);
// x[i] *= scale where scale = 1/sqrt(*norm2) read on the device
cudaError_t launch_normalize(float* x, const double* norm2, size_t len, cudaStream_t s);
// trace entry: out[0] = sqrt(dx2 / xs2), out[1] = dx2 + dy2 (device scalars)
cudaError_t launch_trace_combine(const double* dx2, const double* xs2, const double* dy2,
                                 double* out, cudaStream_t s);
// out = alpha * xx + sum(res) / N
cudaError_t launch_objective_combine(const double* xx, const double* res, int n_res,
                                     double alpha, int N, double* out, cudaStream_t s);
cudaError_t launch_fill_nan(double* p, int count, cudaStream_t s);
// zero several buffers in one launch
constexpr int kZeroSegs = 8;
struct ZeroSegs {
    void* ptr[kZeroSegs];
    size_t bytes[kZeroSegs];
    int count;
};
cudaError_t launch_zero_segments(const ZeroSegs& z, cudaStream_t s);
// storage conversions (store 1 binary16, 2 bfloat16; round to nearest even)
cudaError_t launch_to_store(const float* src, unsigned short* dst, size_t len, int store, cudaStream_t s);
cudaError_t launch_from_store(const unsigned short* src, float* dst, size_t len, int store, cudaStream_t s);
// conjugate gradients with device-side float64 scalars
cudaError_t launch_cg_step1(float* x, float* r, const float* p, const float* q, size_t len,
                            const double* rr, const double* pq, cudaStream_t s);
cudaError_t launch_cg_step2(float* p, const float* r, size_t len, const double* rr_new,
                            const double* rr_old, cudaStream_t s);

}  // namespace mcg
