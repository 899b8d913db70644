// Batched channels: many independent D2Q9 instances (uneven nx x ny, own D,
// rates and row velocity profile) advanced together, with the moments of the
// cross-section mean (Sec. 3.2, Eq. 46-47) reduced every step.
//
// Work unit ("tile"): one instance, 32 consecutive columns and a strip of at
// most tile_rows rows; one warp walks the rows of its strip, keeping the strip's part of the cross-section sum phi-bar(x) = sum_y w_y
// phi(x, y) (trapezoid weights, walls on the nodes) in a register. The moments
// sum_x phi-bar(x) {1, xi, xi^2} are linear in phi-bar, so every tile adds its
// strip's partial moments to a fixed slot (xi = x minus an integer reference
// centre, wrapped to [-nx/2, nx/2)), and a fixed-order pass sums the slots per
// instance: the moments are deterministic, and the strips keep the tiles small
// and even so that no CTA waits long at the per-step barrier.
//
// Two execution modes, chosen by the autotuner:
//   PERSISTENT : one cooperative launch runs K steps; warps take tiles from an
//                atomic counter, and a grid barrier (bounded spin, then
//                LBM_E_TIMEOUT) separates the steps;
//   PER_STEP   : one launch per step (one 32 x 16 block per tile, two nodes per
//                thread) plus one moment-reduction launch.
// Either is captured once into a CUDA graph of K steps and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm_cde.h"
#include "lbm_device.cuh"
#include "lbm_pair.cuh"

namespace lbm {

struct InstDev {
    int nx, ny;
    long long off;        // first cell of this instance in the concatenated cell index
    int bc_lo, bc_hi;
    long long tile0, ntiles;
    long long xref0;      // moment reference centre at step 0 (integer node)
    double vref;          // reference drift per step
    const float* urow;    // [2][ny] or nullptr
    Coef c;
    int tx, tyc;          // 32 x 16 cell tiles of the PER_STEP kernel: columns, rows of tiles
    long long ctile0;     // first cell tile of this instance
    long long cblk0, ncblk;   // 256-column blocks of the moment pass
};

// PER_STEP mode: two nodes per thread, one 32 x 16 cell tile per block; the
// instance constants travel in the kernel parameters (warp-uniform reads from
// the constant bank), so the collision holds no coefficient registers.
struct CK {               // the constants collide<D2Q9> reads
    float meq1, meq2, b1, b2, g7, g8;
    float s[9];
    float A[4], C[4];
};

struct InstK {
    long long off;        // first cell of the instance
    const float* urow;
    int nx, ny, tx;       // tx: column tiles
    int tile0;            // first cell tile of the instance within its launch
    int bc_lo, bc_hi;
    CK c;
};

constexpr int CELL_INST = 160;   // instances per launch (kernel parameters < 32 KB)

struct CellArgs {
    float* buf[2];
    const long long* kdev;
    float* strip;         // [cell tiles][32] column sums of w_y phi over each tile's 16 rows
    long long ncat;
    int ninst;            // instances of this launch
    int tile_base;        // first cell tile of this launch
    int koff;             // this launch computes step *kdev + 1 + koff
    InstK inst[CELL_INST];
};

struct TileDev {
    int inst;
    int x0;       // first column
    int y0, y1;   // row strip [y0, y1)
};

struct BatchArgs {
    const InstDev* inst;
    const TileDev* tiles;
    long long ntiles;
    int ninst;
    long long ncat;           // total cells
    float* buf[2];            // state planes [9][ncat], ping-pong
    double* partials;         // [2][ntiles][3]
    double* moments;          // ring [ring][ninst][3], slot (k - 1) mod ring
    int ring;
    const long long* kdev;    // last completed step t: this launch computes t+1 .. t+nsteps
    int nsteps;               // steps in this launch
    unsigned* counter;        // [2] tile counters (PERSISTENT)
    unsigned* bar_count;
    unsigned* bar_gen;
    int* status;              // device status word (LBM_E_TIMEOUT on a barrier time-out)
    long long spin_limit;     // clock64 cycles a CTA may wait at a barrier
};

__device__ __forceinline__ long long wrap_ll(long long v, long long n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// One warp tile of one step (32 columns x the rows [y0, y1) of one instance):
// pull-stream, walls, collide, store, and the strip's partial moments, summed
// over the warp; lane 0 ends with the sums. No block-level synchronisation:
// the instance constants are read through L1.
__device__ __forceinline__ void warp_tile(const BatchArgs& a, long long t, long long k,
                                          const float* __restrict__ src, float* __restrict__ dst, int lane,
                                          double* m)
{
    const TileDev td = a.tiles[t];
    const InstDev& I = a.inst[td.inst];
    const Coef& cs = I.c;
    const int nx = I.nx, ny = I.ny;
    const long long N = a.ncat;
    const int x = td.x0 + lane;
    const bool live = x < nx;
    const int xc = live ? x : nx - 1;
    const int xs[3] = {xc + 1 == nx ? 0 : xc + 1, xc, xc == 0 ? nx - 1 : xc - 1};
    const long long base = I.off;
    const bool walls = I.bc_lo != BC_PERIODIC;
    float col = 0.f, comp = 0.f;   // Kahan sum of w_y phi over the strip of this column
    // software pipeline: the pulls of row y+1 are requested before row y is computed
    auto pull_row = [&](int y, float* f) {
        const int ys[3] = {y + 1 == ny ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i] = __ldg(src + (long long)i * N + base + (long long)ys[D2Q9::ey(i) + 1] * nx + xs[D2Q9::ex(i) + 1]);
    };
    float fnext[9];
    pull_row(td.y0, fnext);
    for (int y = td.y0; y < td.y1; ++y) {
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fnext[i];
        if (y + 1 < td.y1) pull_row(y + 1, fnext);
        const bool lo = walls && y == 0;
        const bool hi = walls && y == ny - 1;
        if (lo || hi) {
            const int kind = lo ? I.bc_lo : I.bc_hi;
            const long long cell = base + (long long)y * nx + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i)
                if (D2Q9::ey(i) != 0 && ((D2Q9::ey(i) == 1) == lo)) {
                    if (kind == BC_BOUNCE) f[i] = __ldg(src + (long long)opposite<D2Q9>(i) * N + cell);
                    else f[i] = f[mirror_y<D2Q9>(i)];
                }
        }
        float ux = 0.f, uy = 0.f;
        if (I.urow) {
            ux = __ldg(I.urow + y);
            uy = __ldg(I.urow + ny + y);
        }
        const float phi = collide<D2Q9>(f, ux, uy, 0.f, cs);
        if (live) {
            const long long cell = base + (long long)y * nx + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) dst[(long long)i * N + cell] = f[i];
        }
        const float w = (walls && (y == 0 || y == ny - 1)) ? 0.5f : 1.0f;
        const float yv = w * phi - comp;
        const float tv = col + yv;
        comp = (tv - col) - yv;
        col = tv;
    }
    // moments of the strip's phi-bar about the integer reference centre
    const long long cref = I.xref0 + (long long)llround(I.vref * (double)k);
    long long xi = wrap_ll((long long)x - cref, nx);
    if (xi >= (nx + 1) / 2) xi -= nx;
    const double pb = live ? (double)col : 0.0;
    m[0] = pb;
    m[1] = pb * (double)xi;
    m[2] = pb * (double)xi * (double)xi;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m[0] += __shfl_down_sync(0xffffffffu, m[0], off);
        m[1] += __shfl_down_sync(0xffffffffu, m[1], off);
        m[2] += __shfl_down_sync(0xffffffffu, m[2], off);
    }
}

// Moments of step k for every instance: one warp per instance sums the tile
// partials with a fixed lane assignment and a fixed shuffle tree.
__device__ void reduce_moments(const BatchArgs& a, long long k, const double* part)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < a.ninst; i += nw) {
        const InstDev& I = a.inst[i];
        double s0 = 0, s1 = 0, s2 = 0;
        for (long long t = I.tile0 + lane; t < I.tile0 + I.ntiles; t += 32) {
            s0 += part[t * 3 + 0];
            s1 += part[t * 3 + 1];
            s2 += part[t * 3 + 2];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s0 += __shfl_down_sync(0xffffffffu, s0, off);
            s1 += __shfl_down_sync(0xffffffffu, s1, off);
            s2 += __shfl_down_sync(0xffffffffu, s2, off);
        }
        if (lane == 0) {
            double* out = a.moments + (((k - 1) % a.ring) * a.ninst + i) * 3;
            out[0] = s0;
            out[1] = s1;
            out[2] = s2;
        }
    }
}

// Grid barrier with a bounded wait: returns false (and latches LBM_E_TIMEOUT)
// if the other CTAs do not arrive within spin_limit cycles.
__device__ bool grid_barrier(const BatchArgs& a)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* gen = a.bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            *a.bar_count = 0u;
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > a.spin_limit || *((volatile int*)a.status) != 0) {
                    atomicCAS(a.status, 0, (int)LBM_E_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// B_0 sits in buf[0], so B_{k-1} is in buf[(k-1) & 1] and B_k goes to buf[k & 1].
// Every warp takes tiles from the step's counter (lane 0 fetches the next index
// while the current tile runs); a grid barrier closes each step.
__global__ void __launch_bounds__(256, 4) k_batch_persistent(const BatchArgs a)
{
    const int lane = threadIdx.x & 31;
    const long long t0 = *a.kdev;
    for (int s = 0; s < a.nsteps; ++s) {
        const long long k = t0 + 1 + s;
        const float* src = a.buf[(k - 1) & 1];
        float* dst = a.buf[k & 1];
        double* part = a.partials + (long long)(k & 1) * a.ntiles * 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.counter[(k + 1) & 1] = 0u;
        unsigned* ctr = a.counter + (k & 1);
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(ctr, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        while ((long long)t < a.ntiles) {
            unsigned tn = 0;
            if (lane == 0) tn = atomicAdd(ctr, 1u);
            double m[3];
            warp_tile(a, t, k, src, dst, lane, m);
            if (lane == 0) {
                part[(long long)t * 3 + 0] = m[0];
                part[(long long)t * 3 + 1] = m[1];
                part[(long long)t * 3 + 2] = m[2];
            }
            t = __shfl_sync(0xffffffffu, tn, 0);
        }
        if (!grid_barrier(a)) return;
        reduce_moments(a, k, part);
    }
}

// PER_STEP mode step: block t is cell tile t of this launch (32 columns x 16
// rows of one instance). A thread owns the nodes (x, y) and (x, y + 8) and
// evaluates both collisions in paired FP32 arithmetic (lbm_pair.cuh); warp 0
// writes the tile's 32 column sums of w_y phi.
// One 32 x 16 cell tile (tile lt of instance I) of step k: the body of
// k_batch_cells and of the cell-tile persistent kernel. Returns the thread's
// part of its column sum of w_y phi (its two nodes); the callers add the eight
// parts of a column through shared memory.
template <typename IX>
__device__ __forceinline__ float cell_tile(const InstK& I, int lt, long long k, float* const (&buf)[2], long long ncat)
{
    const int nx = I.nx, ny = I.ny;
    const int ty = lt / I.tx;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x = (lt - ty * I.tx) * 32 + lane;
    const int y[2] = {ty * 16 + wy, ty * 16 + 8 + wy};
    const bool xlive = x < nx;
    const bool live[2] = {xlive && y[0] < ny, xlive && y[1] < ny};
    const int xc = min(x, nx - 1);
    const int yc[2] = {min(y[0], ny - 1), min(y[1], ny - 1)};
    const float* __restrict__ src = buf[(k - 1) & 1] + I.off;
    float* __restrict__ dst = buf[k & 1] + I.off;
    const IX N = (IX)ncat;
    const int xs[3] = {xc + 1 == nx ? 0 : xc + 1, xc, xc == 0 ? nx - 1 : xc - 1};
    float f[2][9];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int ys[3] = {yc[h] + 1 == ny ? 0 : yc[h] + 1, yc[h], yc[h] == 0 ? ny - 1 : yc[h] - 1};
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[h][i] = __ldg(src + ((IX)i * N + (IX)ys[D2Q9::ey(i) + 1] * nx + xs[D2Q9::ex(i) + 1]));
    }
    const bool walls = I.bc_lo != BC_PERIODIC;
    bool wall[2] = {false, false};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const bool lo_w = walls && yc[h] == 0, hi_w = walls && yc[h] == ny - 1;
        wall[h] = lo_w || hi_w;
        if (lo_w || hi_w) {
            const int kind = lo_w ? I.bc_lo : I.bc_hi;
            const IX cell = (IX)yc[h] * nx + xc;
#pragma unroll
            for (int i = 0; i < 9; ++i)
                if (D2Q9::ey(i) != 0 && ((D2Q9::ey(i) == 1) == lo_w)) {
                    if (kind == BC_BOUNCE) f[h][i] = __ldg(src + ((IX)opposite<D2Q9>(i) * N + cell));
                    else f[h][i] = f[h][mirror_y<D2Q9>(i)];
                }
        }
    }
    float2 ux = sp2(0.f), uy = sp2(0.f);
    if (I.urow) {
        ux = make_float2(__ldg(I.urow + yc[0]), __ldg(I.urow + yc[1]));
        uy = make_float2(__ldg(I.urow + ny + yc[0]), __ldg(I.urow + ny + yc[1]));
    }
    float2 v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = make_float2(f[0][i], f[1][i]);
    const float2 phi = collide_pair_f32(v, ux, uy, I.c);
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (live[h]) {
            const IX cell = (IX)y[h] * nx + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) dst[(IX)i * N + cell] = h ? v[i].y : v[i].x;
        }
    const float pa = live[0] ? (wall[0] ? __fmul_rn(0.5f, phi.x) : phi.x) : 0.f;
    const float pb = live[1] ? (wall[1] ? __fmul_rn(0.5f, phi.y) : phi.y) : 0.f;
    return pa + pb;
}

// Column sum of the tile's eight row parts (warp 0, in row order)
__device__ __forceinline__ void tile_column_sum(const float (&cs)[8][32], float* __restrict__ strip_out)
{
    const int lane = threadIdx.x & 31;
    float sum = cs[0][lane];
#pragma unroll
    for (int r = 1; r < 8; ++r) sum += cs[r][lane];
    strip_out[lane] = sum;
}

// Shared-memory barriers of the persistent cell-tile kernel (PTX mbarrier):
// arrive, and a wait bounded by `limit` SM cycles that gives up at once when
// the status word already holds an error, latching LBM_E_TIMEOUT otherwise.
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool cbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ void cbar_wait(uint32_t bar, uint32_t parity, int* status, long long limit)
{
    if (cbar_test(bar, parity)) return;
    const long long t0 = clock64();
    while (clock64() - t0 < limit && *((volatile int*)status) == 0)
        if (cbar_test(bar, parity)) return;
    atomicCAS(status, 0, (int)LBM_E_TIMEOUT);
}

template <typename IX>
__global__ void __launch_bounds__(256) k_batch_cells(const __grid_constant__ CellArgs a)
{
    const int t = blockIdx.x;
    int lo = 0, hi = a.ninst - 1;        // instance holding tile t (tile0 ascends)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.inst[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    const InstK& I = a.inst[lo];
    __shared__ float cs[8][32];
    cs[threadIdx.x >> 5][threadIdx.x & 31] = cell_tile<IX>(I, t - I.tile0, *a.kdev + 1 + a.koff, a.buf, a.ncat);
    __syncthreads();
    if (threadIdx.x < 32) tile_column_sum(cs, a.strip + (long long)(a.tile_base + t) * 32);
}

// Eq. 47 moments of step k for PER_STEP mode, two deterministic passes.
// Pass 1: one thread per column x of an instance (256-column blocks, each
// within one instance): phi-bar(x) = FP64 sum of the column's tile sums, then
// phi-bar {1, xi, xi^2}, reduced over the block in a fixed tree to one partial.
// Pass 2: one warp per instance adds its block partials in index order.
__device__ __forceinline__ void col_moments(const BatchArgs& a, long long k, int blk, const float* __restrict__ strip,
                                            const int* __restrict__ cblk_inst, double* __restrict__ cpart)
{
    const int i = cblk_inst[blk];
    const InstDev& I = a.inst[i];
    const long long cref = I.xref0 + (long long)llround(I.vref * (double)k);
    const int nx = I.nx;
    const int x = (blk - (int)I.cblk0) * 256 + threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (x < nx) {
        const float* p = strip + (I.ctile0 + (x >> 5)) * 32 + (x & 31);
        const long long step = (long long)I.tx * 32;
        double pb = 0.0;
        for (int ty = 0; ty < I.tyc; ++ty) pb += (double)p[ty * step];
        long long xi = wrap_ll((long long)x - cref, nx);
        if (xi >= (nx + 1) / 2) xi -= nx;
        const double xd = (double)xi;
        s0 = pb;
        s1 = pb * xd;
        s2 = s1 * xd;
    }
    __shared__ double r[3][256];
    r[0][threadIdx.x] = s0;
    r[1][threadIdx.x] = s1;
    r[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int j = 0; j < 3; ++j) r[j][threadIdx.x] += r[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) cpart[(long long)blk * 3 + threadIdx.x] = r[threadIdx.x][0];
    __syncthreads();   // r is free again for the block's next column block
}

__global__ void __launch_bounds__(256) k_batch_col_moments(const BatchArgs a, const float* __restrict__ strip,
                                                           const int* __restrict__ cblk_inst,
                                                           double* __restrict__ cpart, int koff)
{
    col_moments(a, *a.kdev + 1 + koff, blockIdx.x, strip, cblk_inst, cpart);
}

// Pass 2 for instance i (one warp): block partials added in index order with a
// fixed lane assignment and shuffle tree, written to ring slot (k - 1) mod ring.
__device__ __forceinline__ void inst_moments(const BatchArgs& a, long long k, int i, const double* __restrict__ cpart)
{
    const int lane = threadIdx.x & 31;
    const InstDev& I = a.inst[i];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (long long b = I.cblk0 + lane; b < I.cblk0 + I.ncblk; b += 32) {
        s0 += cpart[b * 3 + 0];
        s1 += cpart[b * 3 + 1];
        s2 += cpart[b * 3 + 2];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, off);
        s1 += __shfl_down_sync(0xffffffffu, s1, off);
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) {
        double* out = a.moments + (((k - 1) % a.ring) * a.ninst + i) * 3;
        out[0] = s0;
        out[1] = s1;
        out[2] = s2;
    }
}

__global__ void __launch_bounds__(256) k_batch_inst_moments(const BatchArgs a, const double* __restrict__ cpart,
                                                            int koff)
{
    const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (i >= a.ninst) return;
    inst_moments(a, *a.kdev + 1 + koff, i, cpart);
}

// PERSISTENT mode on cell tiles (tile height 0): one cooperative launch runs
// the steps of a chunk; each step, the blocks walk the 32 x 16 cell tiles and
// run the PER_STEP arithmetic (two nodes per thread, paired FP32). The two
// moment passes are pipelined behind the cells, so that one bounded grid
// barrier per step suffices: ahead of the cells of step k the grid runs the
// column-moment pass of step k - 1 and the per-instance sums of step k - 2
// (column sums and block partials alternate between two buffers by step
// parity); after the last step, one more barrier separates the last two passes.
// Within a block the tiles' column sums pass through two shared row buffers
// guarded by mbarriers instead of block-wide barriers: every thread arrives on
// the buffer's "full" barrier, warp 0 alone waits there, adds the rows and
// arrives on its "empty" barrier, which the warps wait on before they reuse the
// buffer two tiles later; so warps 1-7 may run up to two tiles ahead of warp 0.
// The instance constants travel by value in the kernel parameters, as for
// k_batch_cells (so at most CELL_INST instances), and every read of them is
// uniform over a block.
struct PersistArgs {
    BatchArgs b;
    const int* tile_inst; // instance of every cell tile
    int nctiles;          // cell tiles in all
    float* strip[2];      // column sums of the even / odd steps of the launch
    const int* cblk_inst;
    int ncblk;
    double* cpart[2];     // block partials of the even / odd steps
    int ninst;
    InstK inst[CELL_INST];   // tile0 = the instance's first cell tile
};

template <typename IX>
__global__ void __launch_bounds__(256, 4) k_batch_persistent_cells(const __grid_constant__ PersistArgs p)
{
    const BatchArgs& a = p.b;
    __shared__ float cs[2][8][32];
    __shared__ __align__(8) unsigned long long cbar[4];   // full[0], full[1], empty[0], empty[1]
    const uint32_t full0 = smem_u32(&cbar[0]), empty0 = smem_u32(&cbar[2]);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * b), "r"(256) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty0 + 8 * b), "r"(32) : "memory");
        }
    }
    __syncthreads();
    const int wy = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned j = 0;   // tiles of this block so far (all steps): buffer j & 1, its use j >> 1
    const long long t0 = *a.kdev;
    const int gw = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((long long)gridDim.x * blockDim.x) >> 5);
    for (int s = 0; s < a.nsteps; ++s) {
        const long long k = t0 + 1 + s;
        // step k - 1: its column sums are complete (barrier of the last iteration)
        if (s >= 1)
            for (int blk = blockIdx.x; blk < p.ncblk; blk += gridDim.x)
                col_moments(a, k - 1, blk, p.strip[(s - 1) & 1], p.cblk_inst, p.cpart[(s - 1) & 1]);
        // step k - 2: its block partials were written before that barrier
        if (s >= 2)
            for (int i = gw; i < a.ninst; i += nw) inst_moments(a, k - 2, i, p.cpart[s & 1]);
        // cell tiles blockIdx.x, blockIdx.x + gridDim.x, ...: equal tiles, so the
        // static split is even to one tile, and no block waits on a counter; the
        // column-sum rows alternate by tile
        float* strip = p.strip[s & 1];
        for (int t = blockIdx.x; t < p.nctiles; t += gridDim.x, ++j) {
            const InstK& I = p.inst[p.tile_inst[t]];
            const float part = cell_tile<IX>(I, t - I.tile0, k, a.buf, a.ncat);
            const unsigned b = j & 1u, use = j >> 1;
            if (use >= 1) cbar_wait(empty0 + 8 * b, (use - 1) & 1u, a.status, a.spin_limit);
            cs[b][wy][lane] = part;
            cbar_arrive(full0 + 8 * b);
            if (wy == 0) {
                cbar_wait(full0 + 8 * b, use & 1u, a.status, a.spin_limit);
                tile_column_sum(cs[b], strip + (long long)t * 32);
                cbar_arrive(empty0 + 8 * b);
            }
        }
        if (!grid_barrier(a)) return;
    }
    const int n = a.nsteps;
    if (n < 1) return;
    const long long kl = t0 + n;
    for (int blk = blockIdx.x; blk < p.ncblk; blk += gridDim.x)
        col_moments(a, kl, blk, p.strip[(n - 1) & 1], p.cblk_inst, p.cpart[(n - 1) & 1]);
    if (n >= 2)
        for (int i = gw; i < a.ninst; i += nw) inst_moments(a, kl - 1, i, p.cpart[n & 1]);
    if (!grid_barrier(a)) return;
    for (int i = gw; i < a.ninst; i += nw) inst_moments(a, kl, i, p.cpart[(n - 1) & 1]);
}

__global__ void k_batch_advance(long long* kdev, int n)
{
    *kdev += n;
}

__global__ void k_batch_init(const InstDev* __restrict__ inst, int ninst, const float* __restrict__ phi0,
                             float* __restrict__ f, long long ncat)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncat;
         c += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = ninst - 1;          // instance holding cell c (offsets ascend)
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (inst[mid].off <= c) lo = mid;
            else hi = mid - 1;
        }
        const InstDev& I = inst[lo];
        const int y = (int)((c - I.off) / I.nx);
        const float ux = I.urow ? I.urow[y] : 0.f, uy = I.urow ? I.urow[I.ny + y] : 0.f;
        float fe[9];
        feq_full<D2Q9>(I.c, phi0[c], ux, uy, 0.f, fe);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[(long long)i * ncat + c] = fe[i];
    }
}

__global__ void k_batch_phi(const float* __restrict__ f, long long ncat, float* __restrict__ out)
{
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncat;
         c += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) s += f[(long long)i * ncat + c];
        out[c] = s;
    }
}

static int occupancy_grid(const void* fn)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 256, 0);
    return std::max(1, per) * sms;
}

// Streams and events of the PER_STEP launches: the moment passes of step k run
// on st2 while the cells of step k + 1 run on the batch's stream.
struct StepStreams {
    cudaStream_t st2;
    cudaEvent_t cells_done;       // recorded after the cell launches of a step
    cudaEvent_t moments_done[2];  // after the moment passes of a step, by step parity
    float* strip2;                // the column sums of the odd steps
};

// rows > 0: PERSISTENT on warp tiles of that height; rows == 0: on cell tiles
static cudaError_t launch_mode(int mode, int rows, const BatchArgs& a, const InstK* cinst, const int* tile_inst,
                               int ninst, long long* kdev,
                               const std::vector<CellArgs>& cells, const std::vector<int>& cell_tiles, int nctiles,
                               float* strip, const int* cblk_inst, int ncblk, double* cpart, cudaStream_t st,
                               const StepStreams& ss)
{
    // 32-bit offsets when the last plane offset 9 ncat fits in 31 bits
    const bool i32 = 9LL * a.ncat < (1LL << 31);
    if (mode == LBM_BATCH_PERSISTENT) {
        // tile counters start at zero for the first step of the launch
        cudaError_t e = cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        if (rows > 0) {
            void* args[] = {(void*)&a};
            e = cudaLaunchCooperativeKernel((const void*)k_batch_persistent,
                                            dim3(occupancy_grid((const void*)k_batch_persistent)), dim3(256), args,
                                            0, st);
        } else {
            PersistArgs p{};
            p.b = a;
            p.tile_inst = tile_inst;
            p.nctiles = nctiles;
            p.strip[0] = strip;
            p.strip[1] = ss.strip2;
            p.cblk_inst = cblk_inst;
            p.ncblk = ncblk;
            p.cpart[0] = cpart;
            p.cpart[1] = cpart + 3LL * ncblk;
            p.ninst = ninst;
            for (int i = 0; i < ninst; ++i) p.inst[i] = cinst[i];
            void* args[] = {(void*)&p};
            const void* fn = i32 ? (const void*)k_batch_persistent_cells<int>
                                 : (const void*)k_batch_persistent_cells<long long>;
            e = cudaLaunchCooperativeKernel(fn, dim3(occupancy_grid(fn)), dim3(256), args, 0, st);
        }
        if (e != cudaSuccess) return e;
        k_batch_advance<<<1, 1, 0, st>>>(kdev, a.nsteps);
        return cudaGetLastError();
    }
    // PER_STEP: step s reads the step index *kdev + 1 + s (one advance at the end),
    // writes its column sums to the strip buffer of its parity, and leaves its two
    // moment passes to st2, so that they overlap the cells of step s + 1; the
    // cells of step s + 2 wait for the moment passes of step s (the strip buffer).
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < a.nsteps && e == cudaSuccess; ++s) {
        float* sb = (s & 1) ? ss.strip2 : strip;
        if (s >= 2) e = cudaStreamWaitEvent(st, ss.moments_done[s & 1], 0);
        for (size_t g = 0; g < cells.size() && e == cudaSuccess; ++g) {
            CellArgs ca = cells[g];
            ca.strip = sb;
            ca.koff = s;
            if (i32) k_batch_cells<int><<<(unsigned)cell_tiles[g], 256, 0, st>>>(ca);
            else k_batch_cells<long long><<<(unsigned)cell_tiles[g], 256, 0, st>>>(ca);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ss.cells_done, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.st2, ss.cells_done, 0);
        if (e != cudaSuccess) break;
        k_batch_col_moments<<<(unsigned)ncblk, 256, 0, ss.st2>>>(a, sb, cblk_inst, cpart, s);
        k_batch_inst_moments<<<(unsigned)((a.ninst + 7) / 8), 256, 0, ss.st2>>>(a, cpart, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ss.moments_done[s & 1], ss.st2);
    }
    if (e != cudaSuccess) return e;
    // the last moment passes (and with them every earlier one) before the advance
    if (a.nsteps > 0) e = cudaStreamWaitEvent(st, ss.moments_done[(a.nsteps - 1) & 1], 0);
    if (e != cudaSuccess) return e;
    k_batch_advance<<<1, 1, 0, st>>>(kdev, a.nsteps);
    return cudaGetLastError();
}

}  // namespace lbm

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct lbm_cde_batch_s {
    lbm_cde_batch_opts o{};
    int n = 0;
    std::vector<lbm::InstDev> inst;
    std::vector<lbm::TileDev> tiles;
    long long ncat = 0;
    lbm::InstDev* inst_dev = nullptr;
    lbm::TileDev* tiles_dev = nullptr;
    float* buf[2] = {nullptr, nullptr};
    double* partials = nullptr;
    double* moments = nullptr;     // ring [chunk][n][3]
    unsigned* sync = nullptr;      // counter[2], bar_count, bar_gen, status, step index (long long)
    int* status = nullptr;
    long long* kdev = nullptr;
    long long t = 0;
    bool ready = false;
    int mode = LBM_BATCH_PERSISTENT;
    int rows = 0;                  // rows per warp tile (PERSISTENT); 0: the cell tiles
    int chunk = 64;                // steps per graph replay
    cudaGraphExec_t graph = nullptr;   // one chunk of steps, built lazily for (mode, rows)
    int graph_key[2] = {-1, -1};
    bool use_graph = true;
    double* stage = nullptr;       // pinned host staging for one chunk of moments
    std::vector<lbm::CellArgs> cells;   // PER_STEP launches (instances in groups of CELL_INST)
    std::vector<lbm::InstK> cinst;      // every instance's constants (cell-tile PERSISTENT mode)
    int* tile_inst = nullptr;           // instance of every cell tile (cell-tile PERSISTENT mode)
    int nctiles = 0;                    // cell tiles in all
    std::vector<int> cell_tiles;        // cell tiles of each launch
    float* strip = nullptr;             // [cell tiles][32] column sums (even steps in PER_STEP mode)
    lbm::StepStreams ss{};              // PER_STEP: moment stream, events, odd-step column sums
    int* cblk_inst = nullptr;           // instance of each 256-column block of the moment pass
    int ncblk = 0;
    double* cpart = nullptr;            // [2][ncblk][3] moment partials (PER_STEP uses the first)
    cudaStream_t st = nullptr;
    std::string err;
};

static thread_local std::string g_batch_err;

static lbm_status bfail(lbm_cde_batch_t b, lbm_status s, const std::string& m)
{
    if (b) b->err = m;
    else g_batch_err = m;
    return s;
}

#define BCK(b, call)                                                                       \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) return bfail(b, LBM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

static void* balloc(lbm_cde_batch_t b, size_t n)
{
    if (b->o.alloc) return b->o.alloc(n ? n : 16, b->o.alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, n ? n : 16) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void bfree(lbm_cde_batch_t b, void* p)
{
    if (!p) return;
    if (b->o.free_) b->o.free_(p, b->o.alloc_ctx);
    else if (!b->o.alloc) cudaFree(p);
}

static void batch_coef(const lbm_cde_channel_desc& d, const double A[4], lbm::Coef& c)
{
    const int model = d.model;
    const double defaults[9] = {1.0, 1.1, 1.1, 0, 1.0, 0, 1.0, 1.2, 1.2};
    double s[15] = {0};
    for (int k = 0; k < 9; ++k) s[k] = std::isnan(d.s[k]) ? defaults[k] : d.s[k];
    if (d.tie_q_rates) {
        s[4] = A[0];
        s[6] = A[3];
    }
    std::memset(&c, 0, sizeof(c));
    for (int k = 0; k < 15; ++k) c.s[k] = (float)s[k];
    for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb) {
            c.A[a * 2 + bb] = (float)A[a * 2 + bb];
            // Eq. 30-31 couplings for MRT-A; the MRT-B models use the unmodified S of Eq. 24
            c.C[a * 2 + bb] = model == LBM_MRT_A
                                  ? (float)((A[a * 2 + bb] / 2.0 - (a == bb ? 1.0 : 0.0)) * s[4 + 2 * bb])
                                  : 0.f;
        }
    // equilibrium: Eq. 37 (MRT-A, B3), Eq. 38 (B1), Eq. 39 (B2); f^eq weights of Eq. 17
    c.meq1 = -2.f;
    c.meq2 = model == LBM_MRT_B1 ? 1.f : 2.f;
    c.b1 = (model == LBM_MRT_B1 || model == LBM_MRT_B2) ? 3.f : 0.f;
    c.b2 = (model == LBM_MRT_B1 || model == LBM_MRT_B2) ? -3.f : 0.f;
    c.g7 = (model == LBM_MRT_B1 || model == LBM_MRT_B2) ? 1.f : 0.f;
    c.g8 = c.g7;
    c.w0 = (float)(20.0 / 36.0);
    c.wa = (float)(8.0 / 144.0);
    c.wd = (float)(8.0 / 144.0);
    c.ka = (float)(48.0 / 144.0);
    c.kd = (float)(12.0 / 144.0);
    c.eps0 = (float)((double)c.w0 + 4.0 * (double)c.wa + 4.0 * (double)c.wd - 1.0);
    lbm::fold_offset_coef(c);
}

static lbm::BatchArgs batch_args(lbm_cde_batch_t b, int nsteps)
{
    lbm::BatchArgs a{};
    a.inst = b->inst_dev;
    a.tiles = b->tiles_dev;
    a.ntiles = (long long)b->tiles.size();
    a.ninst = b->n;
    a.ncat = b->ncat;
    a.buf[0] = b->buf[0];
    a.buf[1] = b->buf[1];
    a.partials = b->partials;
    a.moments = b->moments;
    a.ring = b->chunk;
    a.kdev = b->kdev;
    a.nsteps = nsteps;
    a.counter = b->sync;
    a.bar_count = b->sync + 2;
    a.bar_gen = b->sync + 3;
    a.status = b->status;
    a.spin_limit = b->o.barrier_timeout_cycles;
    return a;
}

static cudaError_t launch_batch(lbm_cde_batch_t b, const lbm::BatchArgs& a)
{
    return lbm::launch_mode(b->mode, b->rows, a, b->cinst.data(), b->tile_inst, b->n, b->kdev, b->cells, b->cell_tiles,
                            b->nctiles,
                            b->strip, b->cblk_inst, b->ncblk, b->cpart, b->st, b->ss);
}

static void drop_graph(lbm_cde_batch_t b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_key[0] = b->graph_key[1] = -1;
}

// Captures one chunk of steps into a graph. The step index and the buffer
// parity live on the device, so the same graph serves every chunk.
static lbm_status ensure_graph(lbm_cde_batch_t b)
{
    if (b->graph && b->graph_key[0] == b->mode && b->graph_key[1] == b->rows) return LBM_OK;
    drop_graph(b);
    cudaStream_t cap = nullptr;
    BCK(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaStream_t keep = b->st;
        b->st = cap;
        lbm::BatchArgs a = batch_args(b, b->chunk);
        cudaError_t le = launch_batch(b, a);
        b->st = keep;
        e = cudaStreamEndCapture(cap, &g);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        b->use_graph = false;     // run chunks with direct launches instead
        return LBM_OK;
    }
    b->graph_key[0] = b->mode;
    b->graph_key[1] = b->rows;
    return LBM_OK;
}

// Warp tiles: 32 columns x a strip of at most b->rows rows (none for rows == 0,
// the cell tiles of the PER_STEP arithmetic).
static lbm_status rebuild_tiles(lbm_cde_batch_t b)
{
    b->tiles.clear();
    for (int i = 0; i < b->n; ++i) {
        b->inst[i].tile0 = (long long)b->tiles.size();
        const int ny = b->inst[i].ny;
        const int nstrip = b->rows > 0 ? (ny + b->rows - 1) / b->rows : 0;
        for (int sidx = 0; sidx < nstrip; ++sidx) {
            // strips of nearly equal height
            const int y0 = (int)((long long)ny * sidx / nstrip);
            const int y1 = (int)((long long)ny * (sidx + 1) / nstrip);
            for (int x0 = 0; x0 < b->inst[i].nx; x0 += 32) b->tiles.push_back({i, x0, y0, y1});
        }
        b->inst[i].ntiles = (long long)b->tiles.size() - b->inst[i].tile0;
    }
    bfree(b, b->tiles_dev);
    bfree(b, b->partials);
    b->tiles_dev = static_cast<lbm::TileDev*>(balloc(b, sizeof(lbm::TileDev) * std::max<size_t>(1, b->tiles.size())));
    b->partials = static_cast<double*>(balloc(b, sizeof(double) * 6 * std::max<size_t>(1, b->tiles.size())));
    if (!b->tiles_dev || !b->partials) return bfail(b, LBM_E_OOM, "tile allocation failed");
    if (!b->tiles.empty())
        BCK(b, cudaMemcpyAsync(b->tiles_dev, b->tiles.data(), sizeof(lbm::TileDev) * b->tiles.size(),
                               cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaMemcpyAsync(b->inst_dev, b->inst.data(), sizeof(lbm::InstDev) * b->n, cudaMemcpyHostToDevice,
                           b->st));
    BCK(b, cudaStreamSynchronize(b->st));
    drop_graph(b);
    return LBM_OK;
}

extern "C" {

lbm_status lbm_cde_batch_opts_init(lbm_cde_batch_opts* o)
{
    if (!o) return bfail(nullptr, LBM_E_ARG, "NULL opts");
    std::memset(o, 0, sizeof(*o));
    o->mode = LBM_BATCH_AUTO;
    o->tile_rows = 0;
    o->graph_steps = 64;
    o->barrier_timeout_cycles = 2000000000LL;
    return LBM_OK;
}

lbm_status lbm_cde_batch_create(const lbm_cde_channel_desc* descs, int32_t n, const lbm_cde_batch_opts* opts,
                                lbm_cde_batch_t* out)
{
    if (!descs || n < 1 || !out) return bfail(nullptr, LBM_E_ARG, "bad argument");
    *out = nullptr;
    lbm_cde_batch_opts o;
    if (opts) o = *opts;
    else lbm_cde_batch_opts_init(&o);
    if ((o.alloc == nullptr) != (o.free_ == nullptr)) return bfail(nullptr, LBM_E_ARG, "alloc/free_ mismatch");
    if (o.tile_rows < 0 || o.tile_rows > 1024) return bfail(nullptr, LBM_E_ARG, "tile_rows in [0, 1024]");
    if (o.graph_steps < 1 || o.graph_steps > 4096) return bfail(nullptr, LBM_E_ARG, "graph_steps in [1, 4096]");
    if (o.barrier_timeout_cycles < 0) return bfail(nullptr, LBM_E_ARG, "negative barrier timeout");
    lbm_cde_batch_t b = new (std::nothrow) lbm_cde_batch_s();
    if (!b) return bfail(nullptr, LBM_E_OOM, "host allocation failed");
    b->o = o;
    b->n = n;
    b->st = static_cast<cudaStream_t>(o.stream);
    b->rows = o.tile_rows == 0 && n > lbm::CELL_INST ? 16 : o.tile_rows;   // cell tiles: <= CELL_INST instances
    b->chunk = o.graph_steps;
    b->mode = o.mode == LBM_BATCH_PER_STEP ? LBM_BATCH_PER_STEP : LBM_BATCH_PERSISTENT;
    b->inst.resize(n);
    long long off = 0;
    for (int i = 0; i < n; ++i) {
        const lbm_cde_channel_desc& d = descs[i];
        if (d.nx < 2 || d.nx > (1 << 24) || d.ny < 3 || d.ny > 65535) {
            delete b;
            return bfail(nullptr, LBM_E_ARG, "instance grid out of range (nx >= 2, 3 <= ny <= 65535)");
        }
        if (d.model < LBM_MRT_A || d.model > LBM_MRT_B3) {
            delete b;
            return bfail(nullptr, LBM_E_ARG, "bad model");
        }
        for (int side = 0; side < 2; ++side) {
            const int k = side ? d.bc_hi_y : d.bc_lo_y;
            if (k != LBM_BC_NOFLUX_NODE && k != LBM_BC_BOUNCEBACK && k != LBM_BC_PERIODIC) {
                delete b;
                return bfail(nullptr, LBM_E_ARG, "batch walls: PERIODIC, NOFLUX_NODE or BOUNCEBACK");
            }
        }
        if ((d.bc_lo_y == LBM_BC_PERIODIC) != (d.bc_hi_y == LBM_BC_PERIODIC)) {
            delete b;
            return bfail(nullptr, LBM_E_ARG, "periodic y needs both faces periodic");
        }
        // A = (3 D + I/2)^-1 (Eq. 36 with the MRT-A factor 1/3); D must be SPD
        const double* D = d.D;
        if (!(D[0] > 0) || !(D[0] * D[3] - D[1] * D[2] > 0) || std::fabs(D[1] - D[2]) > 1e-12 * std::fabs(D[0])) {
            delete b;
            return bfail(nullptr, LBM_E_NOT_SPD, "instance D not symmetric positive definite");
        }
        const double Ai[4] = {3 * D[0] + 0.5, 3 * D[1], 3 * D[2], 3 * D[3] + 0.5};
        const double det = Ai[0] * Ai[3] - Ai[1] * Ai[2];
        const double A[4] = {Ai[3] / det, -Ai[1] / det, -Ai[2] / det, Ai[0] / det};
        lbm::InstDev& I = b->inst[i];
        I.nx = (int)d.nx;
        I.ny = (int)d.ny;
        I.off = off;
        I.bc_lo = d.bc_lo_y;
        I.bc_hi = d.bc_hi_y;
        I.xref0 = (long long)llround(d.x_ref0);
        I.vref = d.x_ref_velocity;
        I.urow = d.u_row_dev;
        batch_coef(d, A, I.c);
        I.tx = (I.nx + 31) / 32;
        I.tyc = (I.ny + 15) / 16;
        I.ctile0 = i ? b->inst[i - 1].ctile0 + (long long)b->inst[i - 1].tx * b->inst[i - 1].tyc : 0;
        I.ncblk = (I.nx + 255) / 256;
        I.cblk0 = i ? b->inst[i - 1].cblk0 + b->inst[i - 1].ncblk : 0;
        off += d.nx * d.ny;
    }
    b->ncat = off;
    const long long ncell_tiles = b->inst[n - 1].ctile0 + (long long)b->inst[n - 1].tx * b->inst[n - 1].tyc;
    if (ncell_tiles >= (1LL << 31) - 1) {
        delete b;
        return bfail(nullptr, LBM_E_ARG, "batch too large");
    }
    b->inst_dev = static_cast<lbm::InstDev*>(balloc(b, sizeof(lbm::InstDev) * n));
    for (int p = 0; p < 2; ++p) b->buf[p] = static_cast<float*>(balloc(b, sizeof(float) * 9 * (size_t)off));
    b->sync = static_cast<unsigned*>(balloc(b, 64));
    b->status = reinterpret_cast<int*>(b->sync + 4);
    b->kdev = reinterpret_cast<long long*>(b->sync + 6);
    b->moments = static_cast<double*>(balloc(b, sizeof(double) * 3 * (size_t)n * b->chunk));
    b->strip = static_cast<float*>(balloc(b, sizeof(float) * 32 * (size_t)ncell_tiles));
    b->ss.strip2 = static_cast<float*>(balloc(b, sizeof(float) * 32 * (size_t)ncell_tiles));
    if (cudaStreamCreateWithFlags(&b->ss.st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ss.cells_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ss.moments_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ss.moments_done[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        lbm_cde_batch_destroy(b);
        return bfail(nullptr, LBM_E_CUDA, "batch stream or event creation failed");
    }
    b->ncblk = (int)(b->inst[n - 1].cblk0 + b->inst[n - 1].ncblk);
    b->cblk_inst = static_cast<int*>(balloc(b, sizeof(int) * (size_t)b->ncblk));
    b->cpart = static_cast<double*>(balloc(b, sizeof(double) * 6 * (size_t)b->ncblk));   // two parities
    if (!b->inst_dev || !b->buf[0] || !b->buf[1] || !b->sync || !b->moments || !b->strip || !b->ss.strip2 ||
        !b->cblk_inst ||
        !b->cpart) {
        lbm_cde_batch_destroy(b);
        return bfail(nullptr, LBM_E_OOM, "batch allocation failed");
    }
    {
        std::vector<int> ci((size_t)b->ncblk);
        for (int i = 0; i < n; ++i)
            for (long long q = 0; q < b->inst[i].ncblk; ++q) ci[(size_t)(b->inst[i].cblk0 + q)] = i;
        cudaMemcpyAsync(b->cblk_inst, ci.data(), sizeof(int) * ci.size(), cudaMemcpyHostToDevice, b->st);
        cudaStreamSynchronize(b->st);
    }
    // PER_STEP launches: instances in groups of CELL_INST, constants by value
    for (int g0 = 0; g0 < n; g0 += lbm::CELL_INST) {
        lbm::CellArgs ca{};
        ca.buf[0] = b->buf[0];
        ca.buf[1] = b->buf[1];
        ca.kdev = b->kdev;
        ca.strip = b->strip;
        ca.ncat = b->ncat;
        ca.ninst = std::min(lbm::CELL_INST, n - g0);
        ca.tile_base = (int)b->inst[g0].ctile0;
        long long tiles = 0;
        for (int j = 0; j < ca.ninst; ++j) {
            const lbm::InstDev& I = b->inst[g0 + j];
            lbm::InstK& K = ca.inst[j];
            K.off = I.off;
            K.urow = I.urow;
            K.nx = I.nx;
            K.ny = I.ny;
            K.tx = I.tx;
            K.tile0 = (int)(I.ctile0 - ca.tile_base);
            K.bc_lo = I.bc_lo;
            K.bc_hi = I.bc_hi;
            K.c.meq1 = I.c.meq1;
            K.c.meq2 = I.c.meq2;
            K.c.b1 = I.c.b1;
            K.c.b2 = I.c.b2;
            K.c.g7 = I.c.g7;
            K.c.g8 = I.c.g8;
            for (int q = 0; q < 9; ++q) K.c.s[q] = I.c.s[q];
            for (int q = 0; q < 4; ++q) K.c.A[q] = I.c.A[q], K.c.C[q] = I.c.C[q];
            tiles += (long long)I.tx * I.tyc;
        }
        b->cells.push_back(ca);
        b->cell_tiles.push_back((int)tiles);
    }
    {
        // the same constants for every instance in one device array, tile0 global
        std::vector<lbm::InstK> all((size_t)n);
        for (size_t g = 0; g < b->cells.size(); ++g)
            for (int j = 0; j < b->cells[g].ninst; ++j) {
                lbm::InstK K = b->cells[g].inst[j];
                K.tile0 += b->cells[g].tile_base;
                all[g * lbm::CELL_INST + j] = K;
            }
        b->nctiles = (int)ncell_tiles;
        std::vector<int> ti((size_t)ncell_tiles);
        for (int i = 0; i < n; ++i)
            for (long long q = 0; q < (long long)b->inst[i].tx * b->inst[i].tyc; ++q) ti[(size_t)(b->inst[i].ctile0 + q)] = i;
        b->cinst = all;
        b->tile_inst = static_cast<int*>(balloc(b, sizeof(int) * ti.size()));
        if (!b->tile_inst) {
            lbm_cde_batch_destroy(b);
            return bfail(nullptr, LBM_E_OOM, "batch allocation failed");
        }
        cudaMemcpyAsync(b->tile_inst, ti.data(), sizeof(int) * ti.size(), cudaMemcpyHostToDevice, b->st);
        cudaStreamSynchronize(b->st);
    }
    cudaMemsetAsync(b->sync, 0, 64, b->st);
    lbm_status s = rebuild_tiles(b);
    if (s != LBM_OK) {
        lbm_cde_batch_destroy(b);
        return bfail(nullptr, s, "tile setup failed");
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_cde_batch_destroy(lbm_cde_batch_t b)
{
    if (!b) return LBM_OK;
    cudaStreamSynchronize(b->st);
    drop_graph(b);
    if (b->stage) cudaFreeHost(b->stage);
    bfree(b, b->inst_dev);
    bfree(b, b->tiles_dev);
    bfree(b, b->partials);
    bfree(b, b->buf[0]);
    bfree(b, b->buf[1]);
    bfree(b, b->sync);
    bfree(b, b->moments);
    bfree(b, b->strip);
    bfree(b, b->ss.strip2);
    if (b->ss.st2) {
        cudaStreamSynchronize(b->ss.st2);
        cudaStreamDestroy(b->ss.st2);
    }
    if (b->ss.cells_done) cudaEventDestroy(b->ss.cells_done);
    for (int p = 0; p < 2; ++p)
        if (b->ss.moments_done[p]) cudaEventDestroy(b->ss.moments_done[p]);
    bfree(b, b->cblk_inst);
    bfree(b, b->cpart);
    bfree(b, b->tile_inst);
    delete b;
    return LBM_OK;
}

lbm_status lbm_cde_batch_cells(lbm_cde_batch_t b, int64_t* ncat)
{
    if (!b || !ncat) return bfail(b, LBM_E_ARG, "NULL argument");
    *ncat = b->ncat;
    return LBM_OK;
}

lbm_status lbm_cde_batch_set_phi(lbm_cde_batch_t b, const float* phi_dev)
{
    if (!b || !phi_dev) return bfail(b, LBM_E_ARG, "NULL argument");
    lbm::k_batch_init<<<152 * 8, 256, 0, b->st>>>(b->inst_dev, b->n, phi_dev, b->buf[0], b->ncat);
    BCK(b, cudaGetLastError());
    BCK(b, cudaMemsetAsync(b->sync, 0, 64, b->st));
    b->t = 0;
    b->ready = true;
    return LBM_OK;
}

lbm_status lbm_cde_batch_get_phi(lbm_cde_batch_t b, float* phi_dev)
{
    if (!b || !phi_dev) return bfail(b, LBM_E_ARG, "NULL argument");
    if (!b->ready) return bfail(b, LBM_E_STATE, "set_phi first");
    lbm::k_batch_phi<<<152 * 8, 256, 0, b->st>>>(b->buf[b->t & 1], b->ncat, phi_dev);
    BCK(b, cudaGetLastError());
    return LBM_OK;
}

// Runs nsteps steps; the moments of every step go to moments_host
// ([nsteps][n][3], may be NULL). Each full chunk replays the captured graph.
lbm_status lbm_cde_batch_run(lbm_cde_batch_t b, int64_t nsteps, double* moments_host)
{
    if (!b || nsteps < 0) return bfail(b, LBM_E_ARG, "bad argument");
    if (!b->ready) return bfail(b, LBM_E_STATE, "set_phi first");
    int64_t done = 0;
    while (done < nsteps) {
        const int len = (int)std::min<int64_t>(b->chunk, nsteps - done);
        const long long first = b->t + 1;      // moments ring slot of step k is (k-1) mod chunk
        if (len == b->chunk && b->use_graph) {
            lbm_status s = ensure_graph(b);
            if (s != LBM_OK) return s;
        }
        if (len == b->chunk && b->use_graph && b->graph) {
            BCK(b, cudaGraphLaunch(b->graph, b->st));
        } else {
            lbm::BatchArgs a = batch_args(b, len);
            BCK(b, launch_batch(b, a));
        }
        if (moments_host) {
            // the ring slots of this chunk form at most two contiguous runs; copy
            // them into pinned staging, then into the caller's array
            if (!b->stage) BCK(b, cudaMallocHost(&b->stage, sizeof(double) * 3 * b->n * b->chunk));
            const size_t row = (size_t)3 * b->n;
            const long long s0 = (first - 1) % b->chunk;
            const long long run1 = std::min<long long>(len, b->chunk - s0);
            BCK(b, cudaMemcpyAsync(b->stage, b->moments + s0 * row, sizeof(double) * row * run1,
                                   cudaMemcpyDeviceToHost, b->st));
            if (run1 < len)
                BCK(b, cudaMemcpyAsync(b->stage + run1 * row, b->moments, sizeof(double) * row * (len - run1),
                                       cudaMemcpyDeviceToHost, b->st));
            BCK(b, cudaStreamSynchronize(b->st));
            std::memcpy(moments_host + done * row, b->stage, sizeof(double) * row * len);
        }
        b->t += len;
        done += len;
    }
    BCK(b, cudaStreamSynchronize(b->st));
    int st = 0;
    BCK(b, cudaMemcpy(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) return bfail(b, (lbm_status)st, "a grid barrier timed out (state is no longer valid)");
    return LBM_OK;
}

// Times candidate execution modes and tile widths on `steps` steps each, then
// keeps the fastest (the state is restored afterwards). Writes the choice to
// *mode_out / *tile_out (may be NULL).
lbm_status lbm_cde_batch_autotune(lbm_cde_batch_t b, int64_t steps, int32_t* mode_out, int32_t* tile_out)
{
    if (!b || steps < 1) return bfail(b, LBM_E_ARG, "bad argument");
    if (!b->ready) return bfail(b, LBM_E_STATE, "set_phi first");
    const size_t sb = sizeof(float) * 9 * (size_t)b->ncat;
    // save the state and step index
    float* save = static_cast<float*>(balloc(b, sb));
    if (!save) return bfail(b, LBM_E_OOM, "autotune buffer allocation failed");
    BCK(b, cudaMemcpyAsync(save, b->buf[b->t & 1], sb, cudaMemcpyDeviceToDevice, b->st));
    const long long t_save = b->t;
    const int modes[2] = {LBM_BATCH_PERSISTENT, LBM_BATCH_PER_STEP};
    const int tws[4] = {0, 8, 16, 32};
    float best = 1e30f;
    int best_mode = b->mode, best_tw = b->rows;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int m : modes)
        for (int tw : tws) {
            if (m == LBM_BATCH_PER_STEP && tw != tws[0]) continue;   // fixed 32 x 16 cell tiles
            if (m == LBM_BATCH_PERSISTENT && tw == 0 && b->n > lbm::CELL_INST) continue;
            b->mode = m;
            if (b->rows != tw) {
                b->rows = tw;
                lbm_status s = rebuild_tiles(b);
                if (s != LBM_OK) return s;
            }
            lbm_status s = lbm_cde_batch_run(b, std::min<int64_t>(steps, b->chunk), nullptr);  // warm
            if (s != LBM_OK) return s;
            cudaEventRecord(e0, b->st);
            s = lbm_cde_batch_run(b, steps, nullptr);
            cudaEventRecord(e1, b->st);
            cudaEventSynchronize(e1);
            if (s != LBM_OK) return s;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_mode = m;
                best_tw = tw;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->mode = best_mode;
    if (b->rows != best_tw) {
        b->rows = best_tw;
        lbm_status s = rebuild_tiles(b);
        if (s != LBM_OK) return s;
    }
    // restore: state into buf[t_save & 1], step index on the device
    BCK(b, cudaMemcpyAsync(b->buf[t_save & 1], save, sb, cudaMemcpyDeviceToDevice, b->st));
    BCK(b, cudaMemcpyAsync(b->kdev, &t_save, sizeof(long long), cudaMemcpyHostToDevice, b->st));
    BCK(b, cudaStreamSynchronize(b->st));
    bfree(b, save);
    b->t = t_save;
    if (mode_out) *mode_out = best_mode;
    if (tile_out) *tile_out = best_tw;
    return LBM_OK;
}

lbm_status lbm_cde_batch_config(lbm_cde_batch_t b, int32_t mode, int32_t tile_rows)
{
    if (!b || (mode != LBM_BATCH_PERSISTENT && mode != LBM_BATCH_PER_STEP) || tile_rows < 0 || tile_rows > 1024)
        return bfail(b, LBM_E_ARG, "bad mode or tile height");
    b->mode = mode;
    if (tile_rows == 0 && b->n > lbm::CELL_INST) tile_rows = 16;   // cell tiles: <= CELL_INST instances
    if (b->rows != tile_rows) {
        b->rows = tile_rows;
        return rebuild_tiles(b);
    }
    return LBM_OK;
}

const char* lbm_cde_batch_last_error(lbm_cde_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
