// K1 warp D_i, K2 transpose-CSR build, K5 transpose gather D_i^T with the
// fused z / zbar / primal-prox epilogue of Algorithm 1 (arXiv 2410.10503,
// Sec. II-A: A_i = A D_i; Algorithm 1 steps (i) and (iii)).
#include "mc_kernels.h"

namespace mcg {

// Bilinear pull-back sample (D x)(r, c); weights are the products
// (1-fr or fr) * (1-fc or fc), rounded once, exactly as stored in the CSR.
__device__ __forceinline__ float warp_sample(const float* __restrict__ x, int n,
                                             const RigidGate* rg, const float* field,
                                             int r, int c)
{
    int r0, c0;
    float fr, fc;
    warp_taps(rg, field, n, r, c, r0, c0, fr, fc);
    const float wr[2] = {1.0f - fr, fr};
    const float wc[2] = {1.0f - fc, fc};
    float acc = 0.0f;
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const int i = r0 + di, j = c0 + dj;
            if (i >= 0 && i < n && j >= 0 && j < n)
                acc = fmaf(__fmul_rn(wr[di], wc[dj]), __ldg(x + (size_t)i * n + j), acc);
        }
    return acc;
}

// Layout mode: a tile of 32 columns x 30 rows of w = D x plus a one-pixel
// halo (33 x 31) is computed into shared memory, then written as
// (w, next - w) pairs into the row-line and the column-line layouts (the halo
// supplies "next"; pixels past the image edge are zero).  The 960 tile and
// 63 halo samples take one thread each of a 1024-thread block, so every
// sample's loads are issued in the same round.  The pair just before each
// line's data, (0, w[0]), is written by the tile that holds position 0.
constexpr int kWarpTileRows = 30;

__device__ __forceinline__ void warp_layouts_block(const WarpArgs& a, int bx, int by, int slot)
{
    __shared__ float w_s[kWarpTileRows + 1][34];
    const int gate = sel_gate(a.sel, slot);
    const int n = a.n;
    const RigidGate* rg = a.rigid ? a.rigid + gate : nullptr;
    const float* field = a.field ? a.field + (size_t)gate * 2 * n * n : nullptr;
    const int r_t = by * kWarpTileRows, c_t = bx * 32;
    const int tid = threadIdx.x;
    {
        // thread -> sample: tile (rows 0..29, columns 0..31), then the halo
        // column 32 (rows 0..30), then the halo row 30 (columns 0..31)
        int rr = -1, cc = 0;
        if (tid < 32 * kWarpTileRows) { rr = tid >> 5; cc = tid & 31; }
        else if (tid < 32 * kWarpTileRows + kWarpTileRows + 1) { rr = tid - 32 * kWarpTileRows; cc = 32; }
        else if (tid < 32 * kWarpTileRows + kWarpTileRows + 33) { rr = kWarpTileRows; cc = tid - (32 * kWarpTileRows + kWarpTileRows + 1); }
        if (rr >= 0) {
            const int r = r_t + rr, c = c_t + cc;
            float w = 0.0f;
            if (r < n && c < n)
                w = a.identity ? __ldg(a.x + (size_t)r * n + c) : warp_sample(a.x, n, rg, field, r, c);
            w_s[rr][cc] = w;
        }
    }
    __syncthreads();
    float2* lrow = a.lrow + slot * a.layout_stride;
    float2* lcol = a.lcol + slot * a.layout_stride;
    if (tid < 32 * kWarpTileRows) {
        {   // row lines: lanes along the columns of one row
            const int rr = tid >> 5, cc = tid & 31;
            const int r = r_t + rr, c = c_t + cc;
            if (r < n && c < n) {
                const float v = w_s[rr][cc];
                lrow[(size_t)r * a.P + a.guard + c] = make_float2(v, w_s[rr][cc + 1] - v);
                if (c == 0) lrow[(size_t)r * a.P + a.guard - 1] = make_float2(0.0f, v);
            }
        }
        {   // column lines: consecutive threads along the rows of one column
            const int cc = tid / kWarpTileRows, rr = tid - cc * kWarpTileRows;
            const int r = r_t + rr, c = c_t + cc;
            if (r < n && c < n) {
                const float v = w_s[rr][cc];
                lcol[(size_t)c * a.P + a.guard + r] = make_float2(v, w_s[rr + 1][cc] - v);
                if (r == 0) lcol[(size_t)c * a.P + a.guard - 1] = make_float2(0.0f, v);
            }
        }
    }
}

__global__ void __launch_bounds__(1024) k_warp_layouts(WarpArgs a)
{
    pdl_wait();
    pdl_trigger();
    warp_layouts_block(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched: the tiles of every slice of the launch, one slice's tile per block.
__global__ void __launch_bounds__(1024) k_warp_layouts_batch(const WarpArgs* __restrict__ args,
                                                             const BatchBlock* __restrict__ map)
{
    pdl_wait();
    pdl_trigger();
    const BatchBlock m = map[blockIdx.x];
    const WarpArgs& a = args[m.slice];
    const int tx = (a.n + 31) / 32;
    warp_layouts_block(a, m.block % tx, m.block / tx, 0);
}

// Plain mode: w = D x as an n x n image.
__global__ void __launch_bounds__(256) k_warp_plain(WarpArgs a)
{
    const int slot = blockIdx.z;
    const int gate = sel_gate(a.sel, slot);
    const int n = a.n;
    const RigidGate* rg = a.rigid ? a.rigid + gate : nullptr;
    const float* field = a.field ? a.field + (size_t)gate * 2 * n * n : nullptr;
    const int c = blockIdx.x * 32 + threadIdx.x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = blockIdx.y * 32 + threadIdx.y + 8 * i;
        if (r < n && c < n)
            a.out[(size_t)slot * n * n + (size_t)r * n + c] =
                a.identity ? __ldg(a.x + (size_t)r * n + c) : warp_sample(a.x, n, rg, field, r, c);
    }
}

cudaError_t launch_warp_layouts(const WarpArgs& a, cudaStream_t s)
{
    if (a.guard < 1 || a.P < a.n + 2 * a.guard) return cudaErrorInvalidValue;   // the lines' zero pairs
    dim3 grid((a.n + 31) / 32, (a.n + kWarpTileRows - 1) / kWarpTileRows, a.n_slots), block(1024);
    return pdl_launch(k_warp_layouts, grid, block, 0, s, a);
}

int warp_layout_tiles(int n) { return ((n + 31) / 32) * ((n + kWarpTileRows - 1) / kWarpTileRows); }

cudaError_t launch_warp_layouts_batch(const WarpArgs* args, const BatchBlock* map, int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    return pdl_launch(k_warp_layouts_batch, dim3(nblocks), dim3(1024), 0, s, args, map);
}

cudaError_t launch_warp_plain(const WarpArgs& a, cudaStream_t s)
{
    dim3 grid((a.n + 31) / 32, (a.n + 31) / 32, a.n_slots), block(32, 8);
    k_warp_plain<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

// ---- K2: CSR of D_i^T: row q lists (p, w) with w the weight of x[q] in (D x)(p)
template <bool FILL>
__global__ void __launch_bounds__(256) k_csr_taps(int n, const RigidGate* rg, const float* field,
                                                  int* cnt, const int* rowptr, int2* ent)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * n) return;
    const int r = p / n, c = p - r * n;
    int r0, c0;
    float fr, fc;
    warp_taps(rg, field, n, r, c, r0, c0, fr, fc);
    const float wr[2] = {1.0f - fr, fr};
    const float wc[2] = {1.0f - fc, fc};
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const int i = r0 + di, j = c0 + dj;
            const float w = __fmul_rn(wr[di], wc[dj]);
            if (i >= 0 && i < n && j >= 0 && j < n && w != 0.0f) {
                const int q = i * n + j;
                if (FILL) {
                    const int pos = rowptr[q] + atomicAdd(cnt + q, 1);
                    ent[pos] = make_int2(p, __float_as_int(w));
                } else {
                    atomicAdd(cnt + q, 1);
                }
            }
        }
}

cudaError_t launch_csr_count(int n, const RigidGate* rg, const float* field, int* cnt,
                             cudaStream_t s)
{
    const int tot = n * n;
    k_csr_taps<false><<<(tot + 255) / 256, 256, 0, s>>>(n, rg, field, cnt, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_csr_fill(int n, const RigidGate* rg, const float* field,
                            const int* rowptr, int* cursor, int2* ent, cudaStream_t s)
{
    const int tot = n * n;
    k_csr_taps<true><<<(tot + 255) / 256, 256, 0, s>>>(n, rg, field, cursor, rowptr, ent);
    return cudaGetLastError();
}

// Rows are short (about four entries); insertion sort by destination pixel
// makes the summation order, and so the result, deterministic.
__global__ void k_csr_sort(int rows, const int* rowptr, int2* ent)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= rows) return;
    const int b = rowptr[q], e = rowptr[q + 1];
    for (int i = b + 1; i < e; ++i) {
        const int2 v = ent[i];
        int j = i - 1;
        while (j >= b && ent[j].x > v.x) { ent[j + 1] = ent[j]; --j; }
        ent[j + 1] = v;
    }
}

cudaError_t launch_csr_sort(int n, const int* rowptr, int2* ent, cudaStream_t s)
{
    const int rows = n * n;
    k_csr_sort<<<(rows + 255) / 256, 256, 0, s>>>(rows, rowptr, ent);
    return cudaGetLastError();
}

// ---- exclusive scan (3 phases, 1024 elements per block) ---------------------
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* sm, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sm[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? sm[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        sm[lane] = wi - w;          // exclusive warp offsets
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    total = sm[32];
    const int r = sm[wid] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_local(const int* in, int* out, int len,
                                                           int* block_sums)
{
    __shared__ int sm[33];
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const int v = (i < len) ? in[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, sm, total);
    if (i < len) out[i] = ex;
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums in place (any count).
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(int* sums, int count, int* grand)
{
    __shared__ int sm[33];
    int carry = 0;
    for (int base = 0; base < count; base += kScanBlock) {
        const int i = base + threadIdx.x;
        const int v = (i < count) ? sums[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sm, total);
        if (i < count) sums[i] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int* out, int len, const int* sums, const int* grand)
{
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < len) out[i] += sums[blockIdx.x];
    if (i == 0) out[len] = *grand;
}

int scan_scratch_len(int len) { return (len + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t launch_exclusive_scan(const int* in, int* out_rowptr, int len, int* scratch,
                                  int scratch_len, cudaStream_t s)
{
    const int nb = (len + kScanBlock - 1) / kScanBlock;
    if (scratch_len < nb + 1) return cudaErrorInvalidValue;
    k_scan_local<<<nb, kScanBlock, 0, s>>>(in, out_rowptr, len, scratch);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(scratch, nb, scratch + nb);
    k_scan_add<<<nb, kScanBlock, 0, s>>>(out_rowptr, len, scratch, scratch + nb);
    return cudaGetLastError();
}

// ---- field VJP ---------------------------------------------------------------
// out0(p) = g(p) d(D_u x)(p)/du_x(p), out1(p) = g(p) d(D_u x)(p)/du_y(p): the
// derivative of the bilinear pull-back sample at q(p) = p + u(p) inside the
// cell that the floor split of q(p) selects (taps outside the image are
// zero).  With g = A^T r this is the gradient of <A D_u x, r> with respect
// to the dense displacement field u of one gate (Sec. II-A).
__global__ void __launch_bounds__(256) k_field_vjp(int n, const float* __restrict__ field,
                                                   const float* __restrict__ x,
                                                   const float* __restrict__ g,
                                                   float* __restrict__ out0,
                                                   float* __restrict__ out1)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n * n) return;
    const int r = p / n, c = p - r * n;
    int r0, c0;
    float fr, fc;
    warp_taps(nullptr, field, n, r, c, r0, c0, fr, fc);
    float v[2][2];
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) {
            const int i = r0 + di, j = c0 + dj;
            v[di][dj] = (i >= 0 && i < n && j >= 0 && j < n) ? __ldg(x + (size_t)i * n + j) : 0.0f;
        }
    const float dcol = fmaf(fr, v[1][1] - v[1][0], __fmul_rn(1.0f - fr, v[0][1] - v[0][0]));
    const float drow = fmaf(fc, v[1][1] - v[0][1], __fmul_rn(1.0f - fc, v[1][0] - v[0][0]));
    const float gp = __ldg(g + p);
    out0[p] = gp * dcol;
    out1[p] = gp * drow;
}

cudaError_t launch_field_vjp(int n, const float* field, const float* x, const float* g,
                             float* out0, float* out1, cudaStream_t s)
{
    const int tot = n * n;
    k_field_vjp<<<(tot + 255) / 256, 256, 0, s>>>(n, field, x, g, out0, out1);
    return cudaGetLastError();
}

// ---- K5 (+K7) -------------------------------------------------------------
template <bool UPDATE>
__device__ __forceinline__ void warp_adjoint_block(const WarpAdjArgs& a, int bx)
{
    const int n2 = a.n * a.n;
    const int q = bx * 256 + threadIdx.x;
    if (q >= n2) return;
    // the update's own operands first: their loads overlap the CSR chain
    float z0 = 0.0f, x0 = 0.0f;
    if (UPDATE) { z0 = a.z[q]; x0 = a.x_in[q]; }
    float v = 0.0f;
    for (int s = 0; s < a.n_slots; ++s) {
        const int gate = sel_gate(a.sel, s);
        const int* rp = a.rowptr + (size_t)gate * (n2 + 1);
        const int2* ent = a.ent + a.ent_off[gate];
        const float* b = a.b + (size_t)s * n2;
        const int e0 = __ldg(rp + q), e1 = __ldg(rp + q + 1);
        int e = e0;
        // four entries per step: their loads and gathers are independent,
        // the accumulation keeps the row's (sorted) order
        for (; e + 4 <= e1; e += 4) {
            const int2 t0 = __ldg(ent + e), t1 = __ldg(ent + e + 1);
            const int2 t2 = __ldg(ent + e + 2), t3 = __ldg(ent + e + 3);
            const float b0 = __ldg(b + t0.x), b1 = __ldg(b + t1.x);
            const float b2 = __ldg(b + t2.x), b3 = __ldg(b + t3.x);
            v = fmaf(__int_as_float(t0.y), b0, v);
            v = fmaf(__int_as_float(t1.y), b1, v);
            v = fmaf(__int_as_float(t2.y), b2, v);
            v = fmaf(__int_as_float(t3.y), b3, v);
        }
        for (; e < e1; ++e) {
            const int2 t = __ldg(ent + e);
            v = fmaf(__int_as_float(t.y), __ldg(b + t.x), v);
        }
    }
    if (UPDATE) {
        // (iii) z^{k+1} = z^k + v, zbar^{k+1} = z^{k+1} + (theta/p_i) v, then
        // (i) of the next iteration: x^{k+2} = (x^{k+1} - tau zbar^{k+1}) / (1 + 2 tau alpha)
        const float zn = z0 + v;
        const float coef = a.coef_tab ? __ldg(a.coef_tab + sel_block(a.sel, 0)) : a.coef;
        const float zbar = fmaf(coef, v, zn);
        a.z[q] = zn;
        a.x_out[q] = fmaf(-a.tau, zbar, x0) * a.prox_scale;
    } else {
        a.out[q] = v;
    }
}

// One warp moves a slice's gate sequence from the iteration of parity t to
// the next (see BatchDraw): the position advances, and at an epoch's end the
// next epoch's gates are drawn into the other half as the one-slice draw does.
__device__ __forceinline__ void advance_gate_sequence(const BatchDraw& d, int t)
{
    int pos = d.state[2 * t] + 1, epar = d.state[2 * t + 1];
    if (pos >= d.n_blocks) {
        pos = 0;
        epar ^= 1;
        const uint64_t k0 = (uint64_t)*d.kctr;
        for (int j = threadIdx.x; j < d.n_blocks; j += 32) {
            const uint32_t w = philox_word0(d.seed, d.stream, k0 + (uint64_t)j);
            int g;
            if (!d.thr) {
                g = (int)(((uint64_t)w * (uint64_t)d.n_blocks) >> 32);
            } else {
                g = 0;
                while (g < d.n_blocks - 1 && (unsigned long long)w >= d.thr[g]) ++g;
            }
            d.gates[epar * d.stride + j] = g;
        }
        __syncwarp();
        if (threadIdx.x == 0) *d.kctr = (unsigned long long)(k0 + (uint64_t)d.n_blocks);
    }
    if (threadIdx.x == 0) {
        d.state[2 * (t ^ 1)] = pos;
        d.state[2 * (t ^ 1) + 1] = epar;
    }
}

template <bool UPDATE>
__global__ void __launch_bounds__(256) k_warp_adjoint(WarpAdjArgs a)
{
    pdl_wait();
    pdl_trigger();
    if (UPDATE && a.draw && blockIdx.x == 0 && threadIdx.x < 32) advance_gate_sequence(*a.draw, a.draw_t);
    warp_adjoint_block<UPDATE>(a, blockIdx.x);
}

// Batched: 256 pixels of one slice per block, every slice of the launch; the
// first warp of each slice's first block advances the slice's gate sequence
// to the next iteration.
__global__ void __launch_bounds__(256) k_warp_adjoint_update_batch(const WarpAdjArgs* __restrict__ args,
                                                                   const BatchBlock* __restrict__ map,
                                                                   const BatchDraw* __restrict__ draw, int t)
{
    pdl_wait();
    pdl_trigger();
    const BatchBlock m = map[blockIdx.x];
    if (m.block == 0 && threadIdx.x < 32) advance_gate_sequence(draw[m.slice], t);
    warp_adjoint_block<true>(args[m.slice], m.block);
}

cudaError_t launch_warp_adjoint_store(const WarpAdjArgs& a, cudaStream_t s)
{
    const int n2 = a.n * a.n;
    return pdl_launch(k_warp_adjoint<false>, dim3((n2 + 255) / 256), dim3(256), 0, s, a);
}

cudaError_t launch_warp_adjoint_update(const WarpAdjArgs& a, cudaStream_t s)
{
    const int n2 = a.n * a.n;
    return pdl_launch(k_warp_adjoint<true>, dim3((n2 + 255) / 256), dim3(256), 0, s, a);
}

int warp_adjoint_blocks(int n) { return (n * n + 255) / 256; }

cudaError_t launch_warp_adjoint_update_batch(const WarpAdjArgs* args, const BatchBlock* map, int nblocks,
                                             const BatchDraw* draw, int t, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    return pdl_launch(k_warp_adjoint_update_batch, dim3(nblocks), dim3(256), 0, s, args, map, draw, t);
}

}  // namespace mcg
