// The operator application y = A sigma (Eq. BIEdiscretized + L + pressure fix)
// and the velocity / effective-viscosity extraction, for every cell of the
// batch at once.
//
// Launch sequence of one application (context stream; the wall discrepancy
// and the proxy strengths run on an auxiliary stream beside the near sum):
//   k_pack_moments  q = sigma w as single-, double- or double-float source records, and
//                   F_b = sum q, tau_b = sum (x - x^c)^perp . q  (one CTA per body)
//   k_near32r/64/df 3x3 near image sum of G^t at every node (Sec. 6.2 step 1): one
//                   launch over the work items (cell, target tile, source split) of
//                   all cells -> partial sums per split
//   k_disc          (auxiliary stream) wall discrepancy of the near sum with the
//                   far-image cancellation (Sec. 6.2 step 2), per (wall point,
//                   split, cell) (its last block per wall point forms
//                   g~ = g0 - g, Sec. 6.2 step 3)
//   k_xi            (auxiliary stream) xi = P g~ per (row, cell) (Sec. 6.2 step 3)
// then, single precision (close.cu):
//   k_alpha32       alpha = -T_0 . n_0 per cell
//   k_assemble32    per target: T = partials + on-curve diagonal + proxy traction
//                   (step 4) + close evaluation (Sec. 6.3) with the own-body and
//                   close pairs redone from positions differenced in double-float;
//                   y = sigma/2 + T + alpha n + L sigma
// or, FP64 and double-float:
//   k_correct       T = sum of partials + on-curve diagonal + proxy traction (step 4)
//   k_close_apply   close-evaluation correction (Sec. 6.3)
//   k_finish        alpha = -T_0 . n_0 per cell;  y = sigma/2 + T + alpha n + L sigma
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "bie_internal.cuh"

namespace bie {

__device__ inline double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double block_sum_d(double v, double* red) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = lane < nw ? red[lane] : 0.0;
        s = warp_sum_d(s);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}


// Knuth's TwoSum: s + e == a + b exactly

// ---------------------------------------------------------------------------


// Work item of a near-sum launch: cell, target tile and source split.  The
// tile covers `tile` targets of the cell; the split covers the cell's sources
// [split * chunk, (split + 1) * chunk), chunk = ceil(N_cell / splits).
struct ItemRange {
    int c, i0, i1, j0, j1, nloc;
    long long out;  // partial base of this split: part_off + split * N_cell - node_off
};

// srcmul: source records per node (1: nodes; 4: the doubled-cell image records).
__device__ __forceinline__ bool item_range(const int4* items, const Cell* cells, int prec, int tile, ItemRange& r,
                                           int srcmul = 1, int item = -1) {
    const int4 it = items[item < 0 ? (int)blockIdx.x : item];
    const Cell& cl = cells[it.x];
    if (!cl.active) return false;
    const int sp = cl.splits[prec];
    const int ns = srcmul * cl.n_nodes;
    // per-node records (srcmul > 1) split at node boundaries: a node's records stay together
    const int chunk = (ns + sp * srcmul - 1) / (sp * srcmul) * srcmul;
    r.c = it.x;
    r.nloc = cl.n_nodes;
    r.i0 = cl.node_off + it.y * tile;
    r.i1 = min(cl.node_off + cl.n_nodes, r.i0 + tile);
    r.j0 = srcmul * cl.node_off + it.z * chunk;
    r.j1 = min(srcmul * cl.node_off + ns, r.j0 + chunk);
    r.out = cl.part_off[prec] + (long long)it.z * cl.n_nodes - cl.node_off;
    return true;
}

// ---------------------------------------------------------------------------
// Near image sum, single precision.  One CTA per work item; kNearThreads
// threads, each owning TPT targets.  The 9 image shifts are applied to the
// target (x_t - s) so every staged source is reused by 9 * TPT pair
// evaluations.  Per pair: 13 FP32 instructions and one MUFU reciprocal.  The
// zero-distance self pair is absorbed by a 1e-30 floor on r^2 (its r.n and
// r.q are exactly zero, so it contributes 0).
// ---------------------------------------------------------------------------
template <int TPT, bool COMP, int MINB>
__global__ void __launch_bounds__(kNearThreads, MINB)
k_near32(const int4* __restrict__ items, const Cell* __restrict__ cells, const float4* __restrict__ tgt,
         const float4* __restrict__ src, float2* __restrict__ part) {
    __shared__ float4 s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 0, kNearThreads * TPT, rg)) return;
    const Cell& cl = cells[rg.c];
    float px[TPT][9], py[TPT][9], nxv[TPT], nyv[TPT];
    float ax[TPT][3], ay[TPT][3];
    // COMP: each source tile's sum is folded into a TwoSum-compensated pair
    // (hi, lo), so that splits with very many sources keep single-precision
    // accuracy relative to the sum instead of losing it to rounding growth.
    float hx[TPT], lx[TPT], hy[TPT], ly[TPT];
    const int tbase = rg.i0 + threadIdx.x;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        int i = tbase + t * kNearThreads;
        float4 tv = i < rg.i1 ? tgt[i] : make_float4(1e4f, 1e4f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            px[t][k] = tv.x - cl.sxf[k];
            py[t][k] = tv.y - cl.syf[k];
        }
        nxv[t] = tv.z;
        nyv[t] = tv.w;
#pragma unroll
        for (int r = 0; r < 3; ++r) ax[t][r] = ay[t][r] = 0.f;
        hx[t] = lx[t] = hy[t] = ly[t] = 0.f;
    }
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < cnt; ++k) {
            float4 s = s_src[k];
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
#pragma unroll
                for (int im = 0; im < 9; ++im) {
                    const float dx = px[t][im] - s.x;
                    const float dy = py[t][im] - s.y;
                    const float cc = pair32(dx, dy, nxv[t], nyv[t], s.z, s.w);
                    ax[t][im / 3] = fmaf(cc, dx, ax[t][im / 3]);
                    ay[t][im / 3] = fmaf(cc, dy, ay[t][im / 3]);
                }
            }
        }
        if constexpr (COMP) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float e;
                float sx_ = (ax[t][0] + ax[t][1]) + ax[t][2];
                float sy_ = (ay[t][0] + ay[t][1]) + ay[t][2];
                two_sum(hx[t], sx_, hx[t], e);
                lx[t] += e;
                two_sum(hy[t], sy_, hy[t], e);
                ly[t] += e;
#pragma unroll
                for (int r = 0; r < 3; ++r) ax[t][r] = ay[t][r] = 0.f;
            }
        }
    }
    const float c = (float)(-1.0 / kPi);
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        int i = tbase + t * kNearThreads;
        if (i < rg.i1) {
            if constexpr (COMP)
                part[rg.out + i] = make_float2(c * (hx[t] + lx[t]), c * (hy[t] + ly[t]));
            else
                part[rg.out + i] =
                    make_float2(c * (ax[t][0] + ax[t][1] + ax[t][2]), c * (ay[t][0] + ay[t][1] + ay[t][2]));
        }
    }
}

// The same sum with two images per packed f32x2 instruction: images
// (0,1), (2,3), (4,5), (6,7) share one packed evaluation, image 8 (the
// unshifted one) is scalar.  Every half performs exactly the scalar
// operations of pair32 in the same order, so each pair's term is bit for bit
// the scalar kernel's (the single-precision close pass relies on that); only
// the grouping of the accumulations differs (lane 0 sums images 0, 2, 4, 6,
// lane 1 images 1, 3, 5, 7, a scalar accumulator image 8).
template <int TPT, bool COMP, int MINB>
__global__ void __launch_bounds__(kNearThreads, MINB)
k_near32x2(const int4* __restrict__ items, const Cell* __restrict__ cells, const float4* __restrict__ tgt,
           const float4* __restrict__ src, float2* __restrict__ part) {
    __shared__ float4 s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 0, kNearThreads * TPT, rg)) return;
    const Cell& cl = cells[rg.c];
    f32x2 px[TPT][4], py[TPT][4], nx2[TPT], ny2[TPT], ax[TPT], ay[TPT];
    float px8[TPT], py8[TPT], nxv[TPT], nyv[TPT], ax8[TPT], ay8[TPT];
    float hx[TPT], lx[TPT], hy[TPT], ly[TPT];
    const f32x2 eps = pk2(1e-30f, 1e-30f), zero = pk2(0.f, 0.f);
    const int tbase = rg.i0 + threadIdx.x;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        const float4 tv = i < rg.i1 ? tgt[i] : make_float4(1e4f, 1e4f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            px[t][p] = pk2(tv.x - cl.sxf[2 * p], tv.x - cl.sxf[2 * p + 1]);
            py[t][p] = pk2(tv.y - cl.syf[2 * p], tv.y - cl.syf[2 * p + 1]);
        }
        px8[t] = tv.x - cl.sxf[8];
        py8[t] = tv.y - cl.syf[8];
        nxv[t] = tv.z;
        nyv[t] = tv.w;
        nx2[t] = pk2(tv.z, tv.z);
        ny2[t] = pk2(tv.w, tv.w);
        ax[t] = ay[t] = zero;
        ax8[t] = ay8[t] = 0.f;
        hx[t] = lx[t] = hy[t] = ly[t] = 0.f;
    }
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        const int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < cnt; ++k) {
            const float4 s = s_src[k];
            const f32x2 sx = pk2(s.x, s.x), sy = pk2(s.y, s.y), qx = pk2(s.z, s.z), qy = pk2(s.w, s.w);
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const f32x2 dx = sub2(px[t][p], sx);
                    const f32x2 dy = sub2(py[t][p], sy);
                    const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, eps));
                    const f32x2 rn = fma2(dx, nx2[t], mul2(dy, ny2[t]));
                    const f32x2 rq = fma2(dx, qx, mul2(dy, qy));
                    float ra, rb;
                    upk2(r2, ra, rb);
                    const f32x2 inv = pk2(rcp_approx(ra), rcp_approx(rb));
                    const f32x2 cc = mul2(mul2(rn, inv), mul2(rq, inv));
                    ax[t] = fma2(cc, dx, ax[t]);
                    ay[t] = fma2(cc, dy, ay[t]);
                }
                const float dx = px8[t] - s.x;
                const float dy = py8[t] - s.y;
                const float cc = pair32(dx, dy, nxv[t], nyv[t], s.z, s.w);
                ax8[t] = fmaf(cc, dx, ax8[t]);
                ay8[t] = fmaf(cc, dy, ay8[t]);
            }
        }
        if constexpr (COMP) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float a0, a1, b0, b1, e;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                two_sum(hx[t], (a0 + a1) + ax8[t], hx[t], e);
                lx[t] += e;
                two_sum(hy[t], (b0 + b1) + ay8[t], hy[t], e);
                ly[t] += e;
                ax[t] = ay[t] = zero;
                ax8[t] = ay8[t] = 0.f;
            }
        }
    }
    const float c = (float)(-1.0 / kPi);
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        if (i < rg.i1) {
            if constexpr (COMP) {
                part[rg.out + i] = make_float2(c * (hx[t] + lx[t]), c * (hy[t] + ly[t]));
            } else {
                float a0, a1, b0, b1;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                part[rg.out + i] = make_float2(c * ((a0 + a1) + ax8[t]), c * ((b0 + b1) + ay8[t]));
            }
        }
    }
}

// The same sum for lattices with e1 = (L1, 0), the time-stepping case
// (Sec. 7): the three images of a lattice row share dy, and with it the
// y-parts of r^2, r.n and r.q (pair32's order), which leaves 9 FP32
// operations per pair and 4 per row instead of 13 per pair.  Rows n = -1
// and n = 0 share the packed f32x2 instructions (one row per half), row
// n = +1 runs scalar; every term is bit for bit pair32's.
template <int TPT, bool COMP>
__device__ __forceinline__ void near32r_item(int item, const int4* __restrict__ items, const Cell* __restrict__ cells,
                                             const float4* __restrict__ tgt, const float4* __restrict__ src,
                                             float2* __restrict__ part) {
    __shared__ float4 s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 0, kNearThreads * TPT, rg, 1, item)) return;
    const Cell& cl = cells[rg.c];
    // per target: packed x for the three columns (halves: rows -1, 0), packed
    // y of the two rows; scalar x of row +1's columns and its y
    f32x2 px[TPT][3], py[TPT], nx2[TPT], ny2[TPT], ax[TPT], ay[TPT];
    float px8[TPT][3], py8[TPT], nxv[TPT], nyv[TPT], ax8[TPT], ay8[TPT];
    float hx[TPT], lx[TPT], hy[TPT], ly[TPT];
    const f32x2 eps = pk2(1e-30f, 1e-30f), zero = pk2(0.f, 0.f);
    const int tbase = rg.i0 + threadIdx.x;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        const float4 tv = i < rg.i1 ? tgt[i] : make_float4(1e4f, 1e4f, 0.f, 0.f);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            px[t][m] = pk2(tv.x - cl.sxf[m], tv.x - cl.sxf[3 + m]);
            px8[t][m] = tv.x - cl.sxf[6 + m];
        }
        py[t] = pk2(tv.y - cl.syf[0], tv.y - cl.syf[3]);
        py8[t] = tv.y - cl.syf[6];
        nxv[t] = tv.z;
        nyv[t] = tv.w;
        nx2[t] = pk2(tv.z, tv.z);
        ny2[t] = pk2(tv.w, tv.w);
        ax[t] = ay[t] = zero;
        ax8[t] = ay8[t] = 0.f;
        hx[t] = lx[t] = hy[t] = ly[t] = 0.f;
    }
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        const int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < cnt; ++k) {
            const float4 s = s_src[k];
            const f32x2 sx = pk2(s.x, s.x), sy = pk2(s.y, s.y), qx = pk2(s.z, s.z), qy = pk2(s.w, s.w);
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const f32x2 dy = sub2(py[t], sy);
                const f32x2 dy2 = fma2(dy, dy, eps);
                const f32x2 dyn = mul2(dy, ny2[t]);
                const f32x2 dyq = mul2(dy, qy);
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const f32x2 dx = sub2(px[t][m], sx);
                    const f32x2 r2 = fma2(dx, dx, dy2);
                    const f32x2 rn = fma2(dx, nx2[t], dyn);
                    const f32x2 rq = fma2(dx, qx, dyq);
                    float ra, rb;
                    upk2(r2, ra, rb);
                    const f32x2 inv = pk2(rcp_approx(ra), rcp_approx(rb));
                    const f32x2 cc = mul2(mul2(rn, inv), mul2(rq, inv));
                    ax[t] = fma2(cc, dx, ax[t]);
                    ay[t] = fma2(cc, dy, ay[t]);
                }
                const float ey = py8[t] - s.y;
                const float ey2 = fmaf(ey, ey, 1e-30f);
                const float eyn = ey * nyv[t];
                const float eyq = ey * s.w;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float dx = px8[t][m] - s.x;
                    const float r2 = fmaf(dx, dx, ey2);
                    const float rn = fmaf(dx, nxv[t], eyn);
                    const float rq = fmaf(dx, s.z, eyq);
                    const float inv = rcp_approx(r2);
                    const float cc = (rn * inv) * (rq * inv);
                    ax8[t] = fmaf(cc, dx, ax8[t]);
                    ay8[t] = fmaf(cc, ey, ay8[t]);
                }
            }
        }
        if constexpr (COMP) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float a0, a1, b0, b1, e;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                two_sum(hx[t], (a0 + a1) + ax8[t], hx[t], e);
                lx[t] += e;
                two_sum(hy[t], (b0 + b1) + ay8[t], hy[t], e);
                ly[t] += e;
                ax[t] = ay[t] = zero;
                ax8[t] = ay8[t] = 0.f;
            }
        }
    }
    const float c = (float)(-1.0 / kPi);
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        if (i < rg.i1) {
            if constexpr (COMP) {
                part[rg.out + i] = make_float2(c * (hx[t] + lx[t]), c * (hy[t] + ly[t]));
            } else {
                float a0, a1, b0, b1;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                part[rg.out + i] = make_float2(c * ((a0 + a1) + ax8[t]), c * ((b0 + b1) + ay8[t]));
            }
        }
    }
}

// One work item per CTA.
template <int TPT, bool COMP, int MINB>
__global__ void __launch_bounds__(kNearThreads, MINB)
k_near32r(const int4* __restrict__ items, const Cell* __restrict__ cells, const float4* __restrict__ tgt,
          const float4* __restrict__ src, float2* __restrict__ part) {
    near32r_item<TPT, COMP>(blockIdx.x, items, cells, tgt, src, part);
}

// Persistent form for batches of uneven cells: a grid of the resident CTA
// slots takes the work items (longest first) from a queue counter, *ctr = 0
// at launch; no CTA ever waits on another.  Each item's partial sums are
// those of k_near32r bit for bit.
template <int TPT, bool COMP, int MINB>
__global__ void __launch_bounds__(kNearThreads, MINB)
k_near32r_queue(const int4* __restrict__ items, int count, int* __restrict__ ctr, const Cell* __restrict__ cells,
                const float4* __restrict__ tgt, const float4* __restrict__ src, float2* __restrict__ part) {
    __shared__ int s_item;
    for (;;) {
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= count) return;
        near32r_item<TPT, COMP>(item, items, cells, tgt, src, part);
    }
}

// Near image sum, double precision (one target per thread).  Same structure;
// the self pair is absorbed by a 1e-300 floor on r^2.
__global__ void __launch_bounds__(kNearThreads)
k_near64(const int4* __restrict__ items, const Cell* __restrict__ cells, const double* __restrict__ x,
         const double* __restrict__ y, const double* __restrict__ nx, const double* __restrict__ ny,
         const Src64* __restrict__ src, double2* __restrict__ part) {
    __shared__ Src64 s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 1, kNearThreads, rg)) return;
    const Cell& cl = cells[rg.c];
    const int i = rg.i0 + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < rg.i1) {
        tx = x[i];
        ty = y[i];
        tnx = nx[i];
        tny = ny[i];
    }
    double px[9], py[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        px[k] = tx - cl.sx[k];
        py[k] = ty - cl.sy[k];
    }
    double ax[3] = {0, 0, 0}, ay[3] = {0, 0, 0};
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            Src64 s = s_src[k];
#pragma unroll
            for (int im = 0; im < 9; ++im) {
                double dx = px[im] - s.x;
                double dy = py[im] - s.y;
                double r2 = fma(dx, dx, fma(dy, dy, 1e-300));
                double rn = fma(dy, tny, dx * tnx);
                double rq = fma(dy, s.w, dx * s.z);
                double inv = 1.0 / r2;
                double cc = (rn * inv) * (rq * inv);
                ax[im / 3] = fma(cc, dx, ax[im / 3]);
                ay[im / 3] = fma(cc, dy, ay[im / 3]);
            }
        }
    }
    if (i < rg.i1) {
        const double c = -1.0 / kPi;
        part[rg.out + i] = make_double2(c * (ax[0] + ax[1] + ax[2]), c * (ay[0] + ay[1] + ay[2]));
    }
}

// ---------------------------------------------------------------------------
// Near image sum in double-float arithmetic ("df64": every quantity is an
// unevaluated sum hi + lo of two floats, ~48 significant bits) on the FP32
// pipe.  GB300's FP64 pipe sustains about 1/100 of the FP32 pair rate, so the
// FP64-accurate refinement residual runs here instead.  Error-free
// transformations: TwoSum (6 FP32 ops) for sums, FMA-based TwoProd (2 ops)
// for products, MUFU rcp refined by one FMA residual step for 1/r^2; the
// difference r = x - y is formed exactly from both words (three TwoSums) and
// r, r.n, r.q are renormalised before they are multiplied, so that the
// dropped lo*lo cross terms stay at 2^-48; each source tile's sum is kept as
// (TwoSum hi, float error) and folded into double accumulators.  About 140
// FP32 instructions per pair; each term is accurate to ~1e-14 of the
// kernel's scale |q| / |r| at any distance (the inputs carry 48 of double's
// 53 bits).
// ---------------------------------------------------------------------------
struct __align__(16) SrcDF {
    float xh, xl, yh, yl, qxh, qxl, qyh, qyl;
};

// (ah + al) * (bh + bl) -> (ph, pl), pl not renormalised
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = ah * bh;
    pl = fmaf(ah, bh, -ph);
    pl = fmaf(ah, bl, fmaf(al, bh, pl));
}


// The y-parts of a double-float pair, shared by every image with the same
// r_y: r_y itself, its square (b + eb) and its products with n_y and q_y.
struct DFy {
    float ryh, ryl, b, eb, pn, en, pq, eq;
};

__device__ __forceinline__ DFy pair_df_y(float pyh, float pyl, float nyh, float nyl, const SrcDF& q) {
    DFy y;
    df_diff(pyh, pyl, q.yh, q.yl, y.ryh, y.ryl);
    y.b = y.ryh * y.ryh;
    y.eb = fmaf(y.ryh, y.ryh, -y.b);
    y.eb = fmaf(y.ryh, y.ryl + y.ryl, y.eb);
    df_mul(y.ryh, y.ryl, nyh, nyl, y.pn, y.en);
    df_mul(y.ryh, y.ryl, q.qyh, q.qyl, y.pq, y.eq);
    return y;
}

// One double-float pair of the near sum from its y-parts: target
// x = pxh + pxl with normal x-component nx, source record q; the term c r,
// c = (r.n / r^2)(r.q / r^2), r = p - y, is added to the tile accumulators
// (TwoSum hi, float error).
__device__ __forceinline__ void pair_df_x(float pxh, float pxl, float nxh, float nxl, const DFy& y, const SrcDF& q,
                                          float& axh, float& axe, float& ayh, float& aye) {
    float rxh, rxl, e;
    const float ryh = y.ryh, ryl = y.ryl;
    df_diff(pxh, pxl, q.xh, q.xl, rxh, rxl);
    // r^2 (the 1e-30 floor absorbs the zero-distance self pair)
    float a, ea, r2h, r2l;
    a = rxh * rxh;
    ea = fmaf(rxh, rxh, -a);
    ea = fmaf(rxh, rxl + rxl, ea);
    two_sum(a, y.b, r2h, e);
    r2l = e + ea + y.eb;
    r2h += 1e-30f;
    // 1 / r^2
    const float ih = rcp_approx(r2h);
    float res = fmaf(-r2h, ih, 1.0f);
    res = fmaf(-r2l, ih, res);
    const float il = ih * res;
    // r . n and r . q
    float p1, e1, rnh, rnl, rqh, rql;
    df_mul(rxh, rxl, nxh, nxl, p1, e1);
    two_sum(p1, y.pn, rnh, e);
    rnl = e + e1 + y.en;
    fast2(rnh, rnl);  // r.n may cancel: renormalise before multiplying
    df_mul(rxh, rxl, q.qxh, q.qxl, p1, e1);
    two_sum(p1, y.pq, rqh, e);
    rql = e + e1 + y.eq;
    fast2(rqh, rql);
    // c = (r.n / r^2) (r.q / r^2), term = c r
    float uh, ul, vh, vl, ch, cl2, th, tl;
    df_mul(rnh, rnl, ih, il, uh, ul);
    df_mul(rqh, rql, ih, il, vh, vl);
    df_mul(uh, ul, vh, vl, ch, cl2);
    df_mul(ch, cl2, rxh, rxl, th, tl);
    two_sum(axh, th, axh, e);
    axe += e + tl;
    df_mul(ch, cl2, ryh, ryl, th, tl);
    two_sum(ayh, th, ayh, e);
    aye += e + tl;
}

// One double-float pair with its own y-parts.
__device__ __forceinline__ void pair_df(float pxh, float pxl, float pyh, float pyl, float nxh, float nxl, float nyh,
                                        float nyl, const SrcDF& q, float& axh, float& axe, float& ayh, float& aye) {
    const DFy y = pair_df_y(pyh, pyl, nyh, nyl, q);
    pair_df_x(pxh, pxl, nxh, nxl, y, q, axh, axe, ayh, aye);
}

// a1 in one pass, one CTA per body: q = sigma w packed into whichever source
// records the application needs (single-precision cell-centred, double,
// double-float), and the body's force and torque moments F_b = sum q,
// tau_b = sum (x - x^c)^perp . q (block reductions in a fixed order).
__global__ void __launch_bounds__(256)
k_pack_moments(const double2* __restrict__ sigma, const double* __restrict__ x, const double* __restrict__ y,
               const double* __restrict__ w, const double* __restrict__ body, const int* __restrict__ body_cell,
               const Cell* __restrict__ cells, float4* __restrict__ src32, Src64* __restrict__ src64,
               SrcDF* __restrict__ srcdf, double* __restrict__ bodyF) {
    __shared__ double red[33];
    const int b = blockIdx.x;
    const double* bd = body + 8 * b;
    const double xc = bd[2], yc = bd[3];
    const int n = (int)bd[5], off = (int)bd[6];
    const Cell& cl = cells[body_cell[b]];
    double fx = 0, fy = 0, tq = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int i = off + k;
        const double2 sg = sigma[i];
        const double wi = w[i], X = x[i], Y = y[i];
        const double qx = sg.x * wi, qy = sg.y * wi;
        fx += qx;
        fy += qy;
        tq += -(Y - yc) * qx + (X - xc) * qy;
        if (src32) src32[i] = make_float4((float)(X - cl.C[0]), (float)(Y - cl.C[1]), (float)qx, (float)qy);
        if (src64) src64[i] = Src64{X, Y, qx, qy};
        if (srcdf) {
            SrcDF r;
            split_df(X - cl.C[0], r.xh, r.xl);
            split_df(Y - cl.C[1], r.yh, r.yl);
            split_df(qx, r.qxh, r.qxl);
            split_df(qy, r.qyh, r.qyl);
            srcdf[i] = r;
        }
    }
    fx = block_sum_d(fx, red);
    fy = block_sum_d(fy, red);
    tq = block_sum_d(tq, red);
    if (threadIdx.x == 0) {
        bodyF[3 * b] = fx;
        bodyF[3 * b + 1] = fy;
        bodyF[3 * b + 2] = tq;
    }
}

__global__ void __launch_bounds__(kNearThreads, 4)
k_near_df(const int4* __restrict__ items, const Cell* __restrict__ cells, const double* __restrict__ x,
          const double* __restrict__ y, const double* __restrict__ nx, const double* __restrict__ ny,
          const SrcDF* __restrict__ src, double2* __restrict__ part) {
    __shared__ SrcDF s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 2, kNearThreads, rg)) return;
    const Cell& cl = cells[rg.c];
    const bool rows = cl.e1[1] == 0.0;
    const int i = rg.i0 + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < rg.i1) {
        tx = x[i] - cl.C[0];
        ty = y[i] - cl.C[1];
        tnx = nx[i];
        tny = ny[i];
    }
    float pxh[9], pxl[9], pyh[9], pyl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        split_df(tx - cl.sx[k], pxh[k], pxl[k]);
        split_df(ty - cl.sy[k], pyh[k], pyl[k]);
    }
    float nxh, nxl, nyh, nyl;
    split_df(tnx, nxh, nxl);
    split_df(tny, nyh, nyl);
    // per tile: hi sums by TwoSum, their errors in a float; folded into double
    // accumulators after every tile so that neither grows with the source count
    double dxs = 0, dys = 0;
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        int cnt = min(kNearTile, rg.j1 - jt);
        float axh = 0, axe = 0, ayh = 0, aye = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const SrcDF q = s_src[k];
            if (rows) {
                // e1 = (L1, 0): the three images of a lattice row share r_y
#pragma unroll
                for (int n = 0; n < 3; ++n) {
                    const DFy yp = pair_df_y(pyh[3 * n], pyl[3 * n], nyh, nyl, q);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        pair_df_x(pxh[3 * n + m], pxl[3 * n + m], nxh, nxl, yp, q, axh, axe, ayh, aye);
                }
            } else {
#pragma unroll
                for (int im = 0; im < 9; ++im)
                    pair_df(pxh[im], pxl[im], pyh[im], pyl[im], nxh, nxl, nyh, nyl, q, axh, axe, ayh, aye);
            }
        }
        dxs += (double)axh + (double)axe;
        dys += (double)ayh + (double)aye;
    }
    if (i < rg.i1) {
        const double c = -1.0 / kPi;
        part[rg.out + i] = make_double2(c * dxs, c * dys);
    }
}

// ---------------------------------------------------------------------------
// The doubled-cell periodizer (n_images 4; Def. Gnear, Sec. 6.2).  Node j
// contributes four image records y_j + (m0 + dm) e1 + (n0 + dn) e2, dm, dn in
// {0, 1} (record 4 j + dm + 2 dn; m0, n0 from its image code), and every
// target is taken at its translate inside U (tgt32, xw, yw), so the near
// sums run over 4 N_cell records with no per-target shifts: 4 N^2 pairs per
// application instead of 9 N^2.
// ---------------------------------------------------------------------------

// a1 for the doubled cell, one CTA per body: q = sigma w, the body moments,
// the per-node records (src64 always; src32n, cell-centred single precision,
// for the single-precision wall discrepancy) and the four image records per
// node in the precision in use.  Record positions are formed as
// (x + shift) - C in double, exactly as the targets' translates, so that a
// node's record at its own translate coincides with its target bit for bit
// (the zero-distance self pair then contributes exactly 0).
__global__ void __launch_bounds__(256)
k_pack_moments_u(const double2* __restrict__ sigma, const double* __restrict__ x, const double* __restrict__ y,
                 const double* __restrict__ w, const double* __restrict__ body, const int* __restrict__ body_cell,
                 const Cell* __restrict__ cells, const int* __restrict__ imc, float4* __restrict__ src32,
                 float4* __restrict__ src32n, Src64* __restrict__ src64, Src64* __restrict__ src64u,
                 SrcDF* __restrict__ srcdf, double* __restrict__ bodyF) {
    __shared__ double red[33];
    const int b = blockIdx.x;
    const double* bd = body + 8 * b;
    const double xc = bd[2], yc = bd[3];
    const int n = (int)bd[5], off = (int)bd[6];
    const Cell& cl = cells[body_cell[b]];
    double fx = 0, fy = 0, tq = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int i = off + k;
        const double2 sg = sigma[i];
        const double wi = w[i], X = x[i], Y = y[i];
        const double qx = sg.x * wi, qy = sg.y * wi;
        fx += qx;
        fy += qy;
        tq += -(Y - yc) * qx + (X - xc) * qy;
        src64[i] = Src64{X, Y, qx, qy};
        const int code = imc[i];
        if (src32n) src32n[i] = make_float4((float)(X - cl.C[0]), (float)(Y - cl.C[1]), (float)qx, (float)qy);
        SrcDF qd;
        if (srcdf) {
            split_df(qx, qd.qxh, qd.qxl);
            split_df(qy, qd.qyh, qd.qyl);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int sh = img_shift(code, r);
            const double PX = X + cl.sx[sh], PY = Y + cl.sy[sh];
            const size_t o = 4 * (size_t)i + r;
            if (src32) src32[o] = make_float4((float)(PX - cl.C[0]), (float)(PY - cl.C[1]), (float)qx, (float)qy);
            if (src64u) src64u[o] = Src64{PX, PY, qx, qy};
            if (srcdf) {
                split_df(PX - cl.C[0], qd.xh, qd.xl);
                split_df(PY - cl.C[1], qd.yh, qd.yl);
                srcdf[o] = qd;
            }
        }
    }
    fx = block_sum_d(fx, red);
    fy = block_sum_d(fy, red);
    tq = block_sum_d(tq, red);
    if (threadIdx.x == 0) {
        bodyF[3 * b] = fx;
        bodyF[3 * b + 1] = fy;
        bodyF[3 * b + 2] = tq;
    }
}

// Single-precision near sum over image records.  Each thread owns TPT
// targets; two consecutive source records share one packed f32x2 evaluation
// (the records are staged in shared memory as separate x, y, qx, qy arrays,
// so a 64-bit load yields the pair), and each half performs exactly the
// operations of pair32 in its order: every pair's term is bit for bit the
// one the single-precision close pass recomputes.  A dummy record (far away,
// zero strength) pads an odd tile.
template <int TPT, bool COMP, int MINB, bool ROWS>
__global__ void __launch_bounds__(kNearThreads, MINB)
k_near32u(const int4* __restrict__ items, const Cell* __restrict__ cells, const float4* __restrict__ tgt,
          const float4* __restrict__ src, float2* __restrict__ part) {
    __shared__ __align__(16) float s_x[kNearTile + 2], s_y[kNearTile + 2], s_qx[kNearTile + 2], s_qy[kNearTile + 2];
    ItemRange rg;
    if (!item_range(items, cells, 0, kNearThreads * TPT, rg, 4)) return;
    f32x2 px[TPT], py[TPT], nx2[TPT], ny2[TPT], ax[TPT], ay[TPT];
    float pys[TPT], nys[TPT];
    float hx[TPT], lx[TPT], hy[TPT], ly[TPT];
    const f32x2 eps = pk2(1e-30f, 1e-30f), zero = pk2(0.f, 0.f);
    const int tbase = rg.i0 + threadIdx.x;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        const float4 tv = i < rg.i1 ? tgt[i] : make_float4(1e4f, 1e4f, 0.f, 0.f);
        px[t] = pk2(tv.x, tv.x);
        py[t] = pk2(tv.y, tv.y);
        nx2[t] = pk2(tv.z, tv.z);
        ny2[t] = pk2(tv.w, tv.w);
        pys[t] = tv.y;
        nys[t] = tv.w;
        ax[t] = ay[t] = zero;
        hx[t] = lx[t] = hy[t] = ly[t] = 0.f;
    }
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        const int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) {
            const float4 v = src[jt + k];
            s_x[k] = v.x;
            s_y[k] = v.y;
            s_qx[k] = v.z;
            s_qy[k] = v.w;
        }
        if (threadIdx.x == 0 && (cnt & 1)) {
            s_x[cnt] = 1e4f;
            s_y[cnt] = 1e4f;
            s_qx[cnt] = 0.f;
            s_qy[cnt] = 0.f;
        }
        __syncthreads();
        if constexpr (ROWS) {
            // e1 = (L1, 0): records 2k and 2k + 1 (a node's images dm = 0, 1 at
            // one dn) have the same y and q, so r_y, r_y^2, r_y n_y and r_y q_y
            // are computed once for both (the same roundings as per record)
#pragma unroll 2
            for (int k = 0; k < cnt; k += 2) {
                const f32x2 sx = *reinterpret_cast<const f32x2*>(s_x + k);
                const float sy = s_y[k], qxs = s_qx[k], qys = s_qy[k];
                const f32x2 qx = pk2(qxs, qxs);
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    const float ey = pys[t] - sy;
                    const float ey2 = fmaf(ey, ey, 1e-30f), eyn = ey * nys[t], eyq = ey * qys;
                    const f32x2 dx = sub2(px[t], sx);
                    const f32x2 r2 = fma2(dx, dx, pk2(ey2, ey2));
                    const f32x2 rn = fma2(dx, nx2[t], pk2(eyn, eyn));
                    const f32x2 rq = fma2(dx, qx, pk2(eyq, eyq));
                    float ra, rb;
                    upk2(r2, ra, rb);
                    const f32x2 inv = pk2(rcp_approx(ra), rcp_approx(rb));
                    const f32x2 cc = mul2(mul2(rn, inv), mul2(rq, inv));
                    ax[t] = fma2(cc, dx, ax[t]);
                    ay[t] = fma2(cc, pk2(ey, ey), ay[t]);
                }
            }
        } else {
#pragma unroll 2
            for (int k = 0; k < cnt; k += 2) {
                const f32x2 sx = *reinterpret_cast<const f32x2*>(s_x + k);
                const f32x2 sy = *reinterpret_cast<const f32x2*>(s_y + k);
                const f32x2 qx = *reinterpret_cast<const f32x2*>(s_qx + k);
                const f32x2 qy = *reinterpret_cast<const f32x2*>(s_qy + k);
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    const f32x2 dx = sub2(px[t], sx);
                    const f32x2 dy = sub2(py[t], sy);
                    const f32x2 r2 = fma2(dx, dx, fma2(dy, dy, eps));
                    const f32x2 rn = fma2(dx, nx2[t], mul2(dy, ny2[t]));
                    const f32x2 rq = fma2(dx, qx, mul2(dy, qy));
                    float ra, rb;
                    upk2(r2, ra, rb);
                    const f32x2 inv = pk2(rcp_approx(ra), rcp_approx(rb));
                    const f32x2 cc = mul2(mul2(rn, inv), mul2(rq, inv));
                    ax[t] = fma2(cc, dx, ax[t]);
                    ay[t] = fma2(cc, dy, ay[t]);
                }
            }
        }
        if constexpr (COMP) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                float a0, a1, b0, b1, e;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                two_sum(hx[t], a0 + a1, hx[t], e);
                lx[t] += e;
                two_sum(hy[t], b0 + b1, hy[t], e);
                ly[t] += e;
                ax[t] = ay[t] = zero;
            }
        }
    }
    const float c = (float)(-1.0 / kPi);
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kNearThreads;
        if (i < rg.i1) {
            if constexpr (COMP) {
                part[rg.out + i] = make_float2(c * (hx[t] + lx[t]), c * (hy[t] + ly[t]));
            } else {
                float a0, a1, b0, b1;
                upk2(ax[t], a0, a1);
                upk2(ay[t], b0, b1);
                part[rg.out + i] = make_float2(c * (a0 + a1), c * (b0 + b1));
            }
        }
    }
}

// Double-precision near sum over image records (one target per thread).
__global__ void __launch_bounds__(kNearThreads)
k_near64u(const int4* __restrict__ items, const Cell* __restrict__ cells, const double* __restrict__ xw,
          const double* __restrict__ yw, const double* __restrict__ nx, const double* __restrict__ ny,
          const Src64* __restrict__ src, double2* __restrict__ part) {
    __shared__ Src64 s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 1, kNearThreads, rg, 4)) return;
    const int i = rg.i0 + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < rg.i1) {
        tx = xw[i];
        ty = yw[i];
        tnx = nx[i];
        tny = ny[i];
    }
    double ax = 0, ay = 0;
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        const int cnt = min(kNearTile, rg.j1 - jt);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const Src64 q = s_src[k];
            const double dx = tx - q.x, dy = ty - q.y;
            const double r2 = fma(dx, dx, fma(dy, dy, 1e-300));
            const double rn = fma(dy, tny, dx * tnx);
            const double rq = fma(dy, q.w, dx * q.z);
            const double inv = 1.0 / r2;
            const double cc = (rn * inv) * (rq * inv);
            ax = fma(cc, dx, ax);
            ay = fma(cc, dy, ay);
        }
    }
    if (i < rg.i1) {
        const double c = -1.0 / kPi;
        part[rg.out + i] = make_double2(c * ax, c * ay);
    }
}

// Double-float near sum over image records (one target per thread).
__global__ void __launch_bounds__(kNearThreads, 4)
k_near_dfu(const int4* __restrict__ items, const Cell* __restrict__ cells, const double* __restrict__ xw,
           const double* __restrict__ yw, const double* __restrict__ nx, const double* __restrict__ ny,
           const SrcDF* __restrict__ src, double2* __restrict__ part) {
    __shared__ SrcDF s_src[kNearTile];
    ItemRange rg;
    if (!item_range(items, cells, 2, kNearThreads, rg, 4)) return;
    const Cell& cl = cells[rg.c];
    const bool rows = cl.e1[1] == 0.0;
    const int i = rg.i0 + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < rg.i1) {
        tx = xw[i] - cl.C[0];
        ty = yw[i] - cl.C[1];
        tnx = nx[i];
        tny = ny[i];
    }
    float pxh, pxl, pyh, pyl, nxh, nxl, nyh, nyl;
    split_df(tx, pxh, pxl);
    split_df(ty, pyh, pyl);
    split_df(tnx, nxh, nxl);
    split_df(tny, nyh, nyl);
    double dxs = 0, dys = 0;
    for (int jt = rg.j0; jt < rg.j1; jt += kNearTile) {
        const int cnt = min(kNearTile, rg.j1 - jt);
        float axh = 0, axe = 0, ayh = 0, aye = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
        if (rows) {
            // e1 = (L1, 0): a node's images dm = 0, 1 at one dn (records 2k,
            // 2k + 1) share their y-parts; the same arithmetic, pair by pair
            for (int k = 0; k + 1 < cnt; k += 2) {
                const DFy yp = pair_df_y(pyh, pyl, nyh, nyl, s_src[k]);
                pair_df_x(pxh, pxl, nxh, nxl, yp, s_src[k], axh, axe, ayh, aye);
                pair_df_x(pxh, pxl, nxh, nxl, yp, s_src[k + 1], axh, axe, ayh, aye);
            }
            if (cnt & 1) pair_df(pxh, pxl, pyh, pyl, nxh, nxl, nyh, nyl, s_src[cnt - 1], axh, axe, ayh, aye);
        } else {
            for (int k = 0; k < cnt; ++k)
                pair_df(pxh, pxl, pyh, pyl, nxh, nxl, nyh, nyl, s_src[k], axh, axe, ayh, aye);
        }
        dxs += (double)axh + (double)axe;
        dys += (double)ayh + (double)aye;
    }
    if (i < rg.i1) {
        const double c = -1.0 / kPi;
        part[rg.out + i] = make_double2(c * dxs, c * dys);
    }
}

// Wall table (per geometry and cell): for each collocation point (L points,
// then D points) the point minus each of its six far-image shifts, the wall
// normal used for the traction and the point itself: 16 doubles (x, y of the
// six points, the normal, the point), then the same 16 values as floats in
// cell-centred coordinates (kWallStride doubles per point).  grid.y = cell.
__global__ void k_wall_table(int m, const double* __restrict__ gl_s, const Cell* __restrict__ cells,
                             const double* __restrict__ e2v, double* __restrict__ wall) {
    const int wp = blockIdx.x * blockDim.x + threadIdx.x, cidx = blockIdx.y;
    if (wp >= 2 * m) return;
    const Cell& cl = cells[cidx];
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = e2v[2 * cidx], e2y = e2v[2 * cidx + 1];
    const double Cx = cl.C[0], Cy = cl.C[1];
    double e1[2] = {e1x, e1y}, e2[2] = {e2x, e2y}, nl[2], nd[2];
    wall_normals(e1, e2, nl, nd);
    const bool isL = wp < m;
    const double s = gl_s[isL ? wp : wp - m];
    double X, Y, ax, ay, bx, by;
    if (isL) {
        X = Cx - 0.5 * e1x + s * e2x;
        Y = Cy - 0.5 * e1y + s * e2y;
        ax = e1x; ay = e1y; bx = e2x; by = e2y;
    } else {
        X = Cx - 0.5 * e2x + s * e1x;
        Y = Cy - 0.5 * e2y + s * e1y;
        ax = e2x; ay = e2y; bx = e1x; by = e1y;
    }
    double* o = wall + ((size_t)cidx * 2 * m + wp) * kWallStride;
    for (int k = -1; k <= 1; ++k) {
        o[2 * (k + 1)] = X - (-2.0 * ax + k * bx);
        o[2 * (k + 1) + 1] = Y - (-2.0 * ay + k * by);
        o[2 * (k + 4)] = X - (ax + k * bx);
        o[2 * (k + 4) + 1] = Y - (ay + k * by);
    }
    o[12] = isL ? nl[0] : nd[0];
    o[13] = isL ? nl[1] : nd[1];
    o[14] = X;  // the collocation point itself (the doubled-cell discrepancy shifts per source)
    o[15] = Y;
    float* of = reinterpret_cast<float*>(o + 16);
    for (int k = 0; k < 12; k += 2) {
        of[k] = (float)(o[k] - Cx);
        of[k + 1] = (float)(o[k + 1] - Cy);
    }
    of[12] = (float)o[12];
    of[13] = (float)o[13];
    of[14] = (float)(X - Cx);
    of[15] = (float)(Y - Cy);
}

int build_wall_table(bie_ctx* c, const double* e2, double* wall, cudaStream_t st) {
    k_wall_table<<<dim3((2 * c->m + 63) / 64, c->ncell), 64, 0, st>>>(c->m, c->gl_s, c->cells, e2, wall);
    BIE_LAUNCH(c, "k_wall_table");
    return BIE_OK;
}

// Wall discrepancy (Sec. 6.2 step 2).  For a collocation point x on L,
//   S_near(x + e1) - S_near(x) = sum_n sum_j [K(x, y_j - 2 e1 + n e2) - K(x, y_j + e1 + n e2)] q_j
// and on D with the roles of e1, e2 exchanged; K is the velocity kernel G or
// the traction kernel G^t with the wall normal.  Block (wp, s, cell): wall
// point wp in [0, 2m) (L points, then D points) of the cell and source split
// s of kDiscSplits; its threads stride over the split's sources and the block
// reduces (u_x, u_y, t_x, t_y) into gpart[((cell * kDiscSplits + s) * 2m + wp) * 4 + comp].
// F32: single precision from the packed cell-centred sources (the inner
// solve's operator); otherwise double precision.
__device__ __forceinline__ float fast_log(float x) { return __logf(x); }
__device__ __forceinline__ double fast_log(double x) { return log(x); }
__device__ __forceinline__ float fast_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

//
// UT (the doubled-cell periodizer): by the same translation invariance a node
// whose images have m in {m0, m0 + 1}, n in {n0, n0 + 1} contributes on L
//   sum_{n = n0, n0 + 1} K(x - (m0 - 1) e1 - n e2, y) - K(x - (m0 + 1) e1 - n e2, y)
// and on D the same with the roles of (m, e1) and (n, e2) exchanged: four
// evaluations per node, each at least half a cell from the wall even when
// the node's body crosses it (the point itself comes from the table; src32
// then holds per-node cell-centred records).
template <bool F32, bool UT>
__global__ void __launch_bounds__(256)
k_disc(const Src64* __restrict__ src64, const float4* __restrict__ src32, const Cell* __restrict__ cells, int m,
       const double* __restrict__ wall, const double* __restrict__ bodyF, double* __restrict__ gpart,
       unsigned int* __restrict__ ticket, double* __restrict__ gt, const int* __restrict__ imc) {
    using Real = typename std::conditional<F32, float, double>::type;
    __shared__ double red[4][8];
    __shared__ bool last;
    const int wp = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y, cidx = blockIdx.z;
    const Cell& cl = cells[cidx];
    if (!cl.active) return;
    // per-geometry table: collocation point minus each of the six far-image
    // shifts (plus images -2a + kb, then minus images a + kb), and the normal;
    // the single-precision path works in cell-centred coordinates
    const double* wt = wall + ((size_t)cidx * 2 * m + wp) * kWallStride;
    Real ox[6], oy[6], n0, n1;
    if constexpr (F32) {
        const float* wf = reinterpret_cast<const float*>(wt + 16);
#pragma unroll
        for (int im = 0; im < 6; ++im) {
            ox[im] = wf[2 * im];
            oy[im] = wf[2 * im + 1];
        }
        n0 = wf[12];
        n1 = wf[13];
    } else {
#pragma unroll
        for (int im = 0; im < 6; ++im) {
            ox[im] = wt[2 * im];
            oy[im] = wt[2 * im + 1];
        }
        n0 = wt[12];
        n1 = wt[13];
    }
    Real ux = 0, uy = 0, tx = 0, ty = 0;
    // the doubled cell: the collocation point, the lattice vectors, and which
    // of them the wall's discrepancy steps along (e1 on L, e2 on D)
    const bool isL = wp < m;
    Real X0, Y0, e1x, e1y, e2x, e2y;
    if constexpr (UT) {
        if constexpr (F32) {
            const float* wf = reinterpret_cast<const float*>(wt + 16);
            X0 = wf[14];
            Y0 = wf[15];
        } else {
            X0 = wt[14];
            Y0 = wt[15];
        }
        e1x = (Real)cl.e1[0];
        e1y = (Real)cl.e1[1];
        e2x = (Real)cl.e2[0];
        e2y = (Real)cl.e2[1];
    }
    const int per = (cl.n_nodes + nsp - 1) / nsp;
    const int j0 = cl.node_off + sp * per, j1 = min(cl.node_off + cl.n_nodes, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        Real sx, sy, qx, qy;
        if constexpr (F32) {
            const float4 q = src32[j];
            sx = q.x; sy = q.y; qx = q.z; qy = q.w;
        } else {
            const Src64 q = src64[j];
            sx = q.x; sy = q.y; qx = q.z; qy = q.w;
        }
        constexpr int NE = UT ? 4 : 6;
        Real px[NE], py[NE];
        if constexpr (UT) {
            const int code = imc[j];
            const int jm0 = img_m0(code), jn0 = img_n0(code);
            // evaluation points x - a e1 - b e2: two plus terms, then two minus terms
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int d = k & 1, sgn = k < 2 ? -1 : 1;
                const int a = isL ? jm0 + sgn : jm0 + d, b = isL ? jn0 + d : jn0 + sgn;
                px[k] = X0 - ((Real)a * e1x + (Real)b * e2x);
                py[k] = Y0 - ((Real)a * e1y + (Real)b * e2y);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                px[k] = ox[k];
                py[k] = oy[k];
            }
        }
#pragma unroll
        for (int im = 0; im < NE; ++im) {
            const Real rx = px[im] - sx, ry = py[im] - sy;
            const Real r2 = rx * rx + ry * ry;
            const Real inv = fast_rcp(r2);
            const Real rq = rx * qx + ry * qy;
            const Real l = (Real)(-0.5) * fast_log(r2);
            const Real a = rq * inv;
            const Real vx = l * qx + rx * a, vy = l * qy + ry * a;
            const Real cc = (rx * n0 + ry * n1) * a * inv;
            if (im < NE / 2) {
                ux += vx; uy += vy; tx += cc * rx; ty += cc * ry;
            } else {
                ux -= vx; uy -= vy; tx -= cc * rx; ty -= cc * ry;
            }
        }
    }
    Real v[4] = {ux, uy, tx, ty};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        Real t = v[c];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[c][warp] = (double)t;
    }
    __syncthreads();
    const size_t nv = 8 * (size_t)m;
    double* gp = gpart + (size_t)cidx * kDiscSplits * nv;
    if (threadIdx.x < 4) {
        double t = 0;
        for (int k = 0; k < nw; ++k) t += red[threadIdx.x][k];
        const double scale = threadIdx.x < 2 ? 1.0 / (4.0 * kPi * cl.mu) : -1.0 / kPi;
        gp[(size_t)sp * nv + 4 * wp + threadIdx.x] = t * scale;
    }
    // the last split of this wall point to finish adds the splits in order
    // and writes the wall point's entries of g~ = g0 - g (Sec. 6.2 step 3),
    // g0 = [0; F / 2|e2|; 0; F / 2|e1|] with F the cell's total force
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket + (size_t)cidx * 2 * m + wp, 1u) == (unsigned)nsp - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        // the cell's total force, by one warp
        double fx = 0, fy = 0;
        for (int b = cl.body_off + lane; b < cl.body_off + cl.n_bodies; b += 32) {
            fx += bodyF[3 * b];
            fy += bodyF[3 * b + 1];
        }
        fx = warp_sum_d(fx);
        fy = warp_sum_d(fy);
        if (lane < 4) {
            const int c = lane;
            double g = 0;
            for (int b = 0; b < nsp; ++b) g += __ldcg(gp + (size_t)b * nv + 4 * wp + c);
            const double f = c == 2 ? fx : fy;
            double* d = gt + (size_t)cidx * nv;
            const bool L = wp < m;  // L: rows of blocks 1 (velocity) and 2 (traction); D: blocks 3 and 4
            const int l = L ? wp : wp - m;
            const int row = (L ? 0 : 4 * m) + c * m + l;
            d[row] = c < 2 ? -g : f / (2.0 * (L ? cl.l2 : cl.l1)) - g;
            if (c == 0) ticket[(size_t)cidx * 2 * m + wp] = 0u;
        }
    }
}

// xi = P g~ (Sec. 6.2 step 3).  One warp-sized CTA per (row r of P, cell):
// GB300's FP64 pipe is narrow, so the compensated products are spread over as
// many SMs as there are rows.  Each row is a compensated dot product (Ogita,
// Rump & Oishi's Dot2: FMA-exact products, error-free sums; P has entries up
// to ~1/lam, so a plain double-precision product would add relative noise
// ~1e-11 to the correction and put a floor under the GMRES residual).  xi is
// also stored in single precision for the single-precision correction.
__global__ void __launch_bounds__(32)
k_xi(const double* __restrict__ gt, int m, int M, const Cell* __restrict__ cells, const double* __restrict__ Pall,
     double* __restrict__ xiall, float* __restrict__ xifall) {
    const int lane = threadIdx.x, r = blockIdx.x, cidx = blockIdx.y;
    if (!cells[cidx].active) return;
    const int nv = 8 * m;
    const double* d = gt + (size_t)cidx * nv;
    const double* P = Pall + (size_t)cidx * 2 * M * nv;
    double s = 0, e = 0;
    for (int cc = lane; cc < nv; cc += 32) {
        const double a = P[(size_t)r * nv + cc], b = d[cc];
        const double p = a * b;
        const double pe = fma(a, b, -p);
        const double t = s + p;
        const double z = t - s;
        e += pe + ((s - (t - z)) + (p - z));
        s = t;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const double e2 = __shfl_xor_sync(0xffffffffu, e, o);
        const double t = s + s2;
        const double z = t - s;
        e = e + e2 + ((s - (t - z)) + (s2 - z));
        s = t;
    }
    if (lane == 0) {
        xiall[(size_t)cidx * 2 * M + r] = s + e;
        xifall[(size_t)cidx * 2 * M + r] = (float)(s + e);
    }
}

// T = near partials + on-curve diagonal -(kappa/2pi) tau (tau . q) + proxy
// traction, double-precision paths.  kCorrLanes lanes per target split the
// near-sum partials and the proxies, then combine with shuffles (fixed order:
// deterministic).
__global__ void __launch_bounds__(256)
k_correct(const double2* __restrict__ part, int prec, int N, const int* __restrict__ node_cell,
          const Cell* __restrict__ cells, const double2* __restrict__ sigma, const double* __restrict__ x,
          const double* __restrict__ y, const double* __restrict__ nx, const double* __restrict__ ny,
          const double* __restrict__ w, const double* __restrict__ kap, const double* __restrict__ ypall,
          const double* __restrict__ xiall, int M, double2* __restrict__ T) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) / kCorrLanes;
    const int sub = threadIdx.x % kCorrLanes;
    const int i = g < N ? g : N - 1;
    const int cidx = node_cell[i];
    const Cell& cl = cells[cidx];
    double tx = 0, ty = 0;
    const int splits = cl.splits[prec];
    const long long base = cl.part_off[prec] + (i - cl.node_off);
    for (int s = sub; s < splits; s += kCorrLanes) {
        const double2 p = part[base + (long long)s * cl.n_nodes];
        tx += p.x;
        ty += p.y;
    }
    const double n0 = nx[i], n1 = ny[i];
    const double* yp = ypall + (size_t)cidx * 2 * M;
    const double* xi = xiall + (size_t)cidx * 2 * M;
    const double X = x[i], Y = y[i];
    double cx = 0, cy = 0;
    for (int p = sub; p < M; p += kCorrLanes) {
        const double rx = X - yp[2 * p], ry = Y - yp[2 * p + 1];
        const double fx = xi[p], fy = xi[M + p];
        const double inv = 1.0 / (rx * rx + ry * ry);
        const double cc = ((rx * n0 + ry * n1) * inv) * ((rx * fx + ry * fy) * inv);
        cx += cc * rx;
        cy += cc * ry;
    }
    tx += -cx / kPi;
    ty += -cy / kPi;
#pragma unroll
    for (int o = kCorrLanes / 2; o > 0; o >>= 1) {
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    if (sub != 0 || g >= N) return;
    const double2 sg = sigma[i];
    const double t0 = -n1, t1 = n0;  // unit tangent
    const double qx = sg.x * w[i], qy = sg.y * w[i];
    const double dg = -(kap[i] / (2.0 * kPi)) * (t0 * qx + t1 * qy);
    T[i] = make_double2(tx + dg * t0, ty + dg * t1);
}

// The same for the single-precision path, on the FP32 pipe: the partials are
// added with TwoSum compensation, the proxy traction uses the cell-centred
// single-precision targets, proxies and strengths; only the per-target
// results and the diagonal term are formed in double.
__global__ void k_finish(const double2* __restrict__ T, const double2* __restrict__ sigma, int N,
                         const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ nx, const double* __restrict__ ny,
                         const int* __restrict__ owner, const double* __restrict__ body,
                         const double* __restrict__ bodyF, const int* __restrict__ node_cell,
                         const Cell* __restrict__ cells, double2* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int i0 = cells[node_cell[i]].node_off;  // node 0 of the cell's first body
    double2 T0 = T[i0];
    double alpha = -(T0.x * nx[i0] + T0.y * ny[i0]);
    int b = owner[i];
    double xc = body[8 * b + 2], yc = body[8 * b + 3];
    double Fx = bodyF[3 * b], Fy = bodyF[3 * b + 1], tq = bodyF[3 * b + 2];
    double2 Ti = T[i], s = sigma[i];
    double ox = 0.5 * s.x + Ti.x + alpha * nx[i] + Fx - (y[i] - yc) * tq;
    double oy = 0.5 * s.y + Ti.y + alpha * ny[i] + Fy + (x[i] - xc) * tq;
    out[i] = make_double2(ox, oy);
}

__global__ void k_rhs(const double* __restrict__ nx, const double* __restrict__ ny,
                      const int* __restrict__ node_cell, const Cell* __restrict__ cells, int N,
                      double2* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Cell& cl = cells[node_cell[i]];
    const double mg = cl.mu * cl.gamma;
    b[i] = make_double2(-mg * ny[i], -mg * nx[i]);
}

// ---------------------------------------------------------------------------
// near-sum work items
// ---------------------------------------------------------------------------
// Tile shape of the doubled-cell single-precision near sum: targets per
// thread and resident CTAs per SM (compile-time overrides for sweeps).
// Measured on GB300 (400-ellipse cell, per launch): 2/6 16.69 ms, 8/4 16.71,
// 8/3 16.89, 4/5 17.15, 4/4 17.32, 4/6 17.32, 6/4 17.51, 2/8 18.41.
#ifndef BIE_NEARU_TPT
#define BIE_NEARU_TPT 2
#endif
#ifndef BIE_NEARU_CTAS
#define BIE_NEARU_CTAS 6
#endif
constexpr int kNearUTpt = BIE_NEARU_TPT, kNearUCtas = BIE_NEARU_CTAS;
// Batches (more than one cell) run the single-precision near sum in its
// persistent queue form (compile-time switch for comparisons).
#ifndef BIE_NEAR_QUEUE
#define BIE_NEAR_QUEUE 1
#endif
constexpr bool kNearQueue = BIE_NEAR_QUEUE != 0;

static int near_tile(int shape32, int prec, bool ut = false) {
    if (prec == 0) return kNearThreads * (ut ? kNearUTpt : kNear32ShapeList[shape32].tpt);
    return kNearThreads;
}
static int near_ctas_per_sm(int shape32, int prec, bool ut = false) {
    if (prec == 0) return ut ? kNearUCtas : kNear32ShapeList[shape32].ctas;
    return prec == 1 ? 5 : 4;
}

// Source splits of every cell for one precision.  All items of one launch
// cost about the same per staged source whatever their targets (masked
// targets still run), so a launch takes about ceil(items / slots) waves of
// the longest item.  For w = 1, 2, ... the cells' splits are sized so that
// their items fill w waves of the resident CTA slots of all SMs (each cell in
// proportion to its share of the pairs), and the w with the least modelled
// time wins: waves x (longest source chunk + a per-item overhead of
// kItemOverhead sources).  Deterministic: no timing is involved.
static constexpr int kItemOverhead = 32;

// srcmul: source records per node (4 for the doubled-cell image records).
static void choose_splits(const std::vector<Cell>& cells, int tile, int slots, std::vector<int>& splits,
                          int srcmul = 1) {
    double W = 0;
    for (const Cell& cl : cells) W += (double)cl.n_nodes * cl.n_nodes;
    double best = 1e300;
    std::vector<int> sp(cells.size());
    for (int w = 1; w <= 16; ++w) {
        long long items = 0;
        int maxchunk = 0;
        for (size_t k = 0; k < cells.size(); ++k) {
            const int n = cells[k].n_nodes, ns = srcmul * n;
            const int tiles = (n + tile - 1) / tile;
            const double share = (double)w * slots * ((double)n * n / W) / tiles;
            const int s = std::max(1, std::min((ns + 63) / 64, (int)share));
            sp[k] = s;
            items += (long long)tiles * s;
            maxchunk = std::max(maxchunk, (ns + s - 1) / s);
        }
        const double cost = (double)((items + slots - 1) / slots) * (maxchunk + kItemOverhead);
        if (cost < best * (1 - 1e-9)) {
            best = cost;
            splits = sp;
        }
    }
}

// Items (cell, target tile, source split) for every precision; also sets each
// cell's splits and partial offsets and uploads the cell table.
// Items of one precision for the context's current single-precision shape.
static int build_near_items_prec(bie_ctx* c, int prec) {
    const int tile = near_tile(c->shape32, prec, c->utilde);
    std::vector<int> splits;
    choose_splits(c->cells_h, tile, near_ctas_per_sm(c->shape32, prec, c->utilde) * c->sms, splits, c->srcmul);
    std::vector<int4> items;
    long long off = 0;
    for (int ci = 0; ci < c->ncell; ++ci) {
        Cell& cl = c->cells_h[ci];
        const int n = cl.n_nodes;
        cl.splits[prec] = splits[ci];
        cl.part_off[prec] = off;
        off += (long long)splits[ci] * n;
        const int tiles = (n + tile - 1) / tile;
        for (int t = 0; t < tiles; ++t) {
            // a target partition (bie_set_partition) keeps the tiles that meet
            // its node range, and the first tile (node 0's traction fixes the
            // pressure); the splits stay those of the whole cell, so every
            // kept target's partial sums are the unpartitioned ones bit for bit
            const int a = cl.node_off + t * tile, b = std::min(cl.node_off + n, a + tile);
            if (c->shard.on && t > 0 && (b <= c->shard.n0 || a >= c->shard.n1)) continue;
            for (int s = 0; s < splits[ci]; ++s) items.push_back(make_int4(ci, t, s, 0));
        }
    }
    // longest items first (a cell's items cost its source chunk each): the
    // order of the launch's CTAs and of the persistent queue
    std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& b) {
        const Cell& ca = c->cells_h[a.x];
        const Cell& cb = c->cells_h[b.x];
        const int la = (c->srcmul * ca.n_nodes + ca.splits[prec] - 1) / ca.splits[prec];
        const int lb = (c->srcmul * cb.n_nodes + cb.splits[prec] - 1) / cb.splits[prec];
        return la > lb;
    });
    const size_t bytes = off * (prec == 0 ? sizeof(float2) : sizeof(double2));
    if (bytes > c->ws.part_bytes) return fail(c, BIE_EINVAL, "near-sum partial buffer too small");
    if (c->near[prec].items) BIE_CUDA(c, cudaFree(c->near[prec].items));
    c->near[prec].items = nullptr;
    BIE_CUDA(c, cudaMalloc((void**)&c->near[prec].items, items.size() * sizeof(int4)));
    BIE_CUDA(c, cudaMemcpy(c->near[prec].items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    c->near[prec].count = (int)items.size();
    return BIE_OK;
}

int build_near_items(bie_ctx* c) {
    for (int prec = 0; prec < 3; ++prec)
        if (int rc = build_near_items_prec(c, prec)) return rc;
    ++c->epoch;
    return upload_cells(c, c->stream);
}

// Bytes of the near-sum partial buffer (largest over the precisions and the
// single-precision shapes the autotuner may pick).
size_t near_part_bytes(const bie_ctx* c) {
    size_t best = 0;
    for (int prec = 0; prec < 3; ++prec)
        for (int sh = 0; sh < (prec == 0 && !c->utilde ? kNear32Shapes : 1); ++sh) {
            std::vector<int> splits;
            choose_splits(c->cells_h, near_tile(sh, prec, c->utilde), near_ctas_per_sm(sh, prec, c->utilde) * c->sms,
                          splits, c->srcmul);
            long long off = 0;
            for (size_t k = 0; k < splits.size(); ++k) off += (long long)splits[k] * c->cells_h[k].n_nodes;
            best = std::max(best, (size_t)off * (prec == 0 ? sizeof(float2) : sizeof(double2)));
        }
    return best;
}

// Elements of the single-precision partial buffer for the current splits.
size_t near_part32_elems(const bie_ctx* c) {
    const Cell& last = c->cells_h.back();
    return (size_t)(last.part_off[0] + (long long)last.splits[0] * last.n_nodes);
}

// queue: the counter of the persistent form (batches), slots its grid size
template <int TPT, int MINB, bool PACKED>
static void near32_variant(bool comp, bool rows, int blocks, cudaStream_t st, const int4* items, const Cell* cells,
                           const float4* tgt, const float4* src, float2* part, int* queue = nullptr, int slots = 0) {
    if (PACKED && rows && queue) {
        cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (comp)
            k_near32r_queue<TPT, true, MINB><<<slots, kNearThreads, 0, st>>>(items, blocks, queue, cells, tgt, src,
                                                                            part);
        else
            k_near32r_queue<TPT, false, MINB><<<slots, kNearThreads, 0, st>>>(items, blocks, queue, cells, tgt, src,
                                                                             part);
    } else if (PACKED && rows) {
        if (comp)
            k_near32r<TPT, true, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
        else
            k_near32r<TPT, false, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
    } else if (PACKED) {
        if (comp)
            k_near32x2<TPT, true, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
        else
            k_near32x2<TPT, false, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
    } else {
        if (comp)
            k_near32<TPT, true, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
        else
            k_near32<TPT, false, MINB><<<blocks, kNearThreads, 0, st>>>(items, cells, tgt, src, part);
    }
}

static int launch_near32(bie_ctx* c, const float4* src, float2* part) {
    const NearItems& it = c->near[0];
    if (it.count == 0) return BIE_OK;
    // splits with many sources keep their accuracy through compensated tile sums
    int maxchunk = 0;
    for (const Cell& cl : c->cells_h)
        maxchunk = std::max(maxchunk, (c->srcmul * cl.n_nodes + cl.splits[0] - 1) / cl.splits[0]);
    const bool comp = maxchunk > kNear32CompChunk;
    // lattice rows share dy when every cell has e1 = (L1, 0)
    bool rows = true;
    for (const Cell& cl : c->cells_h) rows = rows && cl.e1[1] == 0.0;
    if (c->utilde) {
        const dim3 g(it.count), b(kNearThreads);
        if (comp && rows) k_near32u<kNearUTpt, true, kNearUCtas, true><<<g, b, 0, c->stream>>>(it.items, c->cells, c->tgt32, src, part);
        else if (comp) k_near32u<kNearUTpt, true, kNearUCtas, false><<<g, b, 0, c->stream>>>(it.items, c->cells, c->tgt32, src, part);
        else if (rows) k_near32u<kNearUTpt, false, kNearUCtas, true><<<g, b, 0, c->stream>>>(it.items, c->cells, c->tgt32, src, part);
        else k_near32u<kNearUTpt, false, kNearUCtas, false><<<g, b, 0, c->stream>>>(it.items, c->cells, c->tgt32, src, part);
        BIE_LAUNCH(c, "k_near32u");
        return BIE_OK;
    }
    // batches of uneven cells take their items from a queue (longest first)
    int* q = (kNearQueue && c->ncell > 1) ? c->near_ctr : nullptr;
    const int sl = kNear32ShapeList[c->shape32].ctas * c->sms;
    // one case per entry of kNear32ShapeList (packed, targets per thread, CTAs per SM)
    switch (c->shape32) {
        case 0: near32_variant<BIE_NEAR32_TPT, BIE_NEAR32_CTAS, true>(comp, rows, it.count, c->stream, it.items, c->cells, c->tgt32, src, part, q, sl); break;
        case 1: near32_variant<1, 8, true>(comp, rows, it.count, c->stream, it.items, c->cells, c->tgt32, src, part, q, sl); break;
        case 2: near32_variant<3, 4, true>(comp, rows, it.count, c->stream, it.items, c->cells, c->tgt32, src, part, q, sl); break;
        case 3: near32_variant<3, 4, false>(comp, rows, it.count, c->stream, it.items, c->cells, c->tgt32, src, part); break;
        default: near32_variant<2, 5, false>(comp, rows, it.count, c->stream, it.items, c->cells, c->tgt32, src, part); break;
    }
    BIE_LAUNCH(c, "k_near32");
    return BIE_OK;
}
#define BIE_SHAPE_IS(k, p, t, m) \
    (kNear32ShapeList[k].packed == (p) && kNear32ShapeList[k].tpt == (t) && kNear32ShapeList[k].ctas == (m))
static_assert(kNear32Shapes == 5 && BIE_SHAPE_IS(0, 1, BIE_NEAR32_TPT, BIE_NEAR32_CTAS) && BIE_SHAPE_IS(1, 1, 1, 8) && BIE_SHAPE_IS(2, 1, 3, 4) &&
                  BIE_SHAPE_IS(3, 0, 3, 4) && BIE_SHAPE_IS(4, 0, 2, 5),
              "launch_near32's cases must match kNear32ShapeList");
#undef BIE_SHAPE_IS

// ---------------------------------------------------------------------------
// One operator application in three parts: 0 pack the sources and body
// moments, 1 the near sum (the part the profiler brackets with events),
// 2 wall discrepancy, proxy fit and correction, close evaluation, assembly.
// a3 + a4: the wall discrepancy g~ of the packed sources and the proxy
// strengths xi = P g~ on stream st (independent of the near sum)
static int launch_disc_xi(bie_ctx* c, bool f32, Workspace& ws, cudaStream_t st) {
    const dim3 dgrid(2 * c->m, kDiscSplits, c->ncell);
    if (c->utilde) {
        if (f32)
            k_disc<true, true><<<dgrid, 256, 0, st>>>(ws.src64, ws.src32n, c->cells, c->m, c->wall, ws.bodyF, ws.gpart,
                                                      ws.dticket, ws.gt, c->imc);
        else
            k_disc<false, true><<<dgrid, 256, 0, st>>>(ws.src64, nullptr, c->cells, c->m, c->wall, ws.bodyF, ws.gpart,
                                                       ws.dticket, ws.gt, c->imc);
    } else if (f32) {
        k_disc<true, false><<<dgrid, 256, 0, st>>>(ws.src64, ws.src32, c->cells, c->m, c->wall, ws.bodyF, ws.gpart,
                                                   ws.dticket, ws.gt, nullptr);
    } else {
        k_disc<false, false><<<dgrid, 256, 0, st>>>(ws.src64, nullptr, c->cells, c->m, c->wall, ws.bodyF, ws.gpart,
                                                    ws.dticket, ws.gt, nullptr);
    }
    BIE_LAUNCH(c, "k_disc");
    k_xi<<<dim3(2 * c->M, c->ncell), 32, 0, st>>>(ws.gt, c->m, c->M, c->cells, c->P, ws.xi, ws.xif);
    BIE_LAUNCH(c, "k_xi");
    return BIE_OK;
}

// One operator application in four parts: 0 packs the sources and body
// moments, 1 is the near sum, 2 the wall discrepancy and proxy strengths
// (independent of 1), 3 the assembly (traction, close evaluation, pressure
// fix, rigid completion).
static int apply_part(bie_ctx* c, int part, const double* sigma, double* yout, int precision, Workspace& ws) {
    const int N = c->N;
    const int bs = 256, gs = (N + bs - 1) / bs;
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    const bool f32 = precision == BIE_MIXED;
    const bool df = precision == BIE_DF64;
    const int prec = f32 ? 0 : (df ? 2 : 1);
    if (part == 0) {
        if (&ws == &c->ws) c->ws_x = nullptr;  // the workspace is about to change
        if (c->utilde)
            k_pack_moments_u<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->body_cell, c->cells,
                                                           c->imc, f32 ? ws.src32 : nullptr, f32 ? ws.src32n : nullptr,
                                                           ws.src64, (!f32 && !df) ? ws.src64u : nullptr,
                                                           df ? (SrcDF*)ws.srcdf : nullptr, ws.bodyF);
        else
            k_pack_moments<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->body_cell, c->cells,
                                                         f32 ? ws.src32 : nullptr, ws.src64,
                                                         df ? (SrcDF*)ws.srcdf : nullptr, ws.bodyF);
        BIE_LAUNCH(c, "k_pack_moments");
        return BIE_OK;
    }
    if (part == 1) {
        if (f32) return launch_near32(c, ws.src32, (float2*)ws.part);
        if (c->utilde) {
            if (df)
                k_near_dfu<<<c->near[2].count, kNearThreads, 0, c->stream>>>(c->near[2].items, c->cells, c->xw, c->yw,
                                                                             c->nx, c->ny, (const SrcDF*)ws.srcdf,
                                                                             (double2*)ws.part);
            else
                k_near64u<<<c->near[1].count, kNearThreads, 0, c->stream>>>(c->near[1].items, c->cells, c->xw, c->yw,
                                                                            c->nx, c->ny, ws.src64u,
                                                                            (double2*)ws.part);
            BIE_LAUNCH(c, df ? "k_near_dfu" : "k_near64u");
            return BIE_OK;
        }
        if (df) {
            k_near_df<<<c->near[2].count, kNearThreads, 0, c->stream>>>(c->near[2].items, c->cells, c->x, c->y,
                                                                        c->nx, c->ny, (const SrcDF*)ws.srcdf,
                                                                        (double2*)ws.part);
            BIE_LAUNCH(c, "k_near_df");
        } else {
            k_near64<<<c->near[1].count, kNearThreads, 0, c->stream>>>(c->near[1].items, c->cells, c->x, c->y, c->nx,
                                                                       c->ny, ws.src64, (double2*)ws.part);
            BIE_LAUNCH(c, "k_near64");
        }
        return BIE_OK;
    }
    if (part == 2) return launch_disc_xi(c, f32, ws, c->stream);
    if (f32) return assemble32(c, sigma, ws, yout);
    double2* T = reinterpret_cast<double2*>(ws.T);
    const int gsc = (N * kCorrLanes + 255) / 256;
    k_correct<<<gsc, 256, 0, c->stream>>>((const double2*)ws.part, prec, N, c->node_cell, c->cells, sg, c->xw, c->yw,
                                          c->nx, c->ny, c->w, c->kap, c->yp, ws.xi, c->M, T);
    BIE_LAUNCH(c, "k_correct");
    if (int rc = close_apply(c, sigma, ws.T)) return rc;
    k_finish<<<gs, bs, 0, c->stream>>>(T, sg, N, c->x, c->y, c->nx, c->ny, c->owner, c->body, ws.bodyF, c->node_cell,
                                       c->cells, reinterpret_cast<double2*>(yout));
    BIE_LAUNCH(c, "k_finish");
    // an FP64-class application over every cell leaves the double-precision
    // sources, body moments and proxy strengths of sigma in the workspace
    if (&ws == &c->ws) {
        bool all = true;
        for (const Cell& cl : c->cells_h) all = all && cl.active;
        if (all) c->ws_x = sigma;
    }
    return BIE_OK;
}

static int apply_impl(bie_ctx* c, const double* sigma, double* yout, int precision, Workspace& ws) {
    const int kind = precision == BIE_MIXED ? 0 : (precision == BIE_DF64 ? 2 : 1);
    if (int rc = apply_part(c, 0, sigma, yout, precision, ws)) return rc;
    // part 2 on the auxiliary stream, overlapping the near sum
    BIE_CUDA(c, cudaEventRecord(c->aux_fork, c->stream));
    BIE_CUDA(c, cudaStreamWaitEvent(c->aux, c->aux_fork, 0));
    if (int rc = launch_disc_xi(c, precision == BIE_MIXED, ws, c->aux)) return rc;
    BIE_CUDA(c, cudaEventRecord(c->aux_join, c->aux));
    if (int rc = prof_begin(c, kind)) return rc;
    if (int rc = apply_part(c, 1, sigma, yout, precision, ws)) return rc;
    if (int rc = prof_end(c)) return rc;
    BIE_CUDA(c, cudaStreamWaitEvent(c->stream, c->aux_join, 0));
    return apply_part(c, 3, sigma, yout, precision, ws);
}

// The single-precision application replayed from CUDA graphs (opts.graph):
// the parts of apply_part are captured once per epoch (any change of their
// arguments: geometry, proxy fit, close pairs, work items) as three graphs
// (pack with the wall discrepancy and proxy strengths; near sum; assembly)
// with fixed input and output buffers, on a stream of the context's own (the
// caller's stream may be the legacy default stream, which cannot capture).
// Each application copies sigma in, replays the graphs on the context's
// stream -- with the profiler's events around the near sum, between the
// graphs, as for direct launches -- and copies the result out.  The same
// kernels with the same inputs (part 2 runs before the near sum instead of
// beside it): the results are bit for bit those of the direct launches.
static int apply_graph(bie_ctx* c, const double* sigma, double* yout) {
    auto& g = c->graph;
    const size_t bytes = 2 * (size_t)c->N * sizeof(double);
    if (!g.in) {
        BIE_CUDA(c, cudaMalloc((void**)&g.in, bytes));
        BIE_CUDA(c, cudaMalloc((void**)&g.out, bytes));
        BIE_CUDA(c, cudaStreamCreateWithFlags(&g.capture, cudaStreamNonBlocking));
    }
    if (!g.exec[0] || g.epoch != c->epoch) {
        for (auto& e : g.exec)
            if (e) {
                BIE_CUDA(c, cudaGraphExecDestroy(e));
                e = nullptr;
            }
        cudaStream_t user = c->stream;
        c->stream = g.capture;
        const long long l0 = c->launches;
        int rc = BIE_OK;
        cudaError_t e = cudaSuccess;
        for (int part = 0; part < 3 && !rc && e == cudaSuccess; ++part) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(g.capture, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            // graphs: pack + wall discrepancy and proxy strengths; near sum; assembly
            static constexpr int kFirst[3] = {0, 1, 3};
            rc = apply_part(c, kFirst[part], g.in, g.out, BIE_MIXED, c->ws);
            if (!rc && part == 0) rc = apply_part(c, 2, g.in, g.out, BIE_MIXED, c->ws);
            e = cudaStreamEndCapture(g.capture, &graph);
            if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec[part], graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        c->stream = user;
        g.kernels = c->launches - l0;
        c->launches = l0;
        if (rc || e != cudaSuccess) {
            for (auto& x : g.exec)
                if (x) {
                    cudaGraphExecDestroy(x);
                    x = nullptr;
                }
            return rc ? rc : cuda_check(c, e, "graph capture");
        }
        g.epoch = c->epoch;
    }
    c->ws_x = nullptr;
    BIE_CUDA(c, cudaMemcpyAsync(g.in, sigma, bytes, cudaMemcpyDeviceToDevice, c->stream));
    BIE_CUDA(c, cudaGraphLaunch(g.exec[0], c->stream));
    if (int rc = prof_begin(c, 0)) return rc;
    BIE_CUDA(c, cudaGraphLaunch(g.exec[1], c->stream));
    if (int rc = prof_end(c)) return rc;
    BIE_CUDA(c, cudaGraphLaunch(g.exec[2], c->stream));
    BIE_CUDA(c, cudaMemcpyAsync(yout, g.out, bytes, cudaMemcpyDeviceToDevice, c->stream));
    c->launches += g.kernels;
    return BIE_OK;
}

void free_graph(bie_ctx* c) {
    auto& g = c->graph;
    for (auto& e : g.exec)
        if (e) cudaGraphExecDestroy(e);
    if (g.in) cudaFree(g.in);
    if (g.out) cudaFree(g.out);
    if (g.capture) cudaStreamDestroy(g.capture);
    for (auto& e : g.exec) e = nullptr;
    g.in = g.out = nullptr;
    g.capture = nullptr;
}

int apply_device(bie_ctx* c, const double* sigma, double* yout, int precision) {
    int rc = (precision == BIE_MIXED && c->opts.graph) ? apply_graph(c, sigma, yout)
                                                       : apply_impl(c, sigma, yout, precision, c->ws);
    if (rc || !c->shard.on) return rc;
    // sharded by target: this process's rows are final; the exchange fills
    // the others from the processes that own them before anything reads them
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->shard.exchange(yout, 2 * (int64_t)c->N, c->shard.user) != 0)
        return fail(c, BIE_ECUDA, "target-partition exchange failed");
    return BIE_OK;
}

// Time every single-precision tile shape on the context's own cells and keep
// the fastest (opts.autotune).  The sources are packed from the right-hand
// side (the work does not depend on the values); per shape one warm-up and
// three timed launches, the median kept.  The shape decides the source splits
// and so the rounding of the single-precision sums: contexts tuned to
// different shapes agree to single-precision accuracy, not bit for bit.
int autotune_near32(bie_ctx* c) {
    const int N = c->N;
    k_rhs<<<(N + 255) / 256, 256, 0, c->stream>>>(c->nx, c->ny, c->node_cell, c->cells, N,
                                                  reinterpret_cast<double2*>(c->sv.r));
    BIE_LAUNCH(c, "k_rhs");
    if (int rc = apply_impl(c, c->sv.r, c->sv.d, BIE_MIXED, c->ws)) return rc;  // packs ws.src32
    cudaEvent_t ev[2];
    BIE_CUDA(c, cudaEventCreate(&ev[0]));
    BIE_CUDA(c, cudaEventCreate(&ev[1]));
    auto ck = [c](cudaError_t e, const char* what) { return e == cudaSuccess ? BIE_OK : cuda_check(c, e, what); };
    int best = 0;
    int rc = BIE_OK;
    for (int sh = 0; sh < kNear32Shapes && !rc; ++sh) {
        c->shape32 = sh;
        if ((rc = build_near_items_prec(c, 0)) || (rc = upload_cells(c, c->stream))) break;
        float t[3];
        for (int k = 0; k < 4 && !rc; ++k) {
            if (k > 0) rc = ck(cudaEventRecord(ev[0], c->stream), "cudaEventRecord");
            if (!rc) rc = launch_near32(c, c->ws.src32, (float2*)c->ws.part);
            if (!rc && k > 0) {
                rc = ck(cudaEventRecord(ev[1], c->stream), "cudaEventRecord");
                if (!rc) rc = ck(cudaEventSynchronize(ev[1]), "cudaEventSynchronize");
                if (!rc) rc = ck(cudaEventElapsedTime(&t[k - 1], ev[0], ev[1]), "cudaEventElapsedTime");
            }
        }
        if (rc) break;
        std::sort(t, t + 3);
        c->tune_ms[sh] = t[1];
        if (t[1] < c->tune_ms[best]) best = sh;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    c->shape32 = best;
    if ((rc = build_near_items_prec(c, 0))) return rc;
    ++c->epoch;
    return upload_cells(c, c->stream);
}

// The single-precision-pair operator application with every per-call buffer
// taken from `ws` (used by the allocation-free entry point, whose buffers
// live in a static device array).  Of the context only the launch counter
// and, with profiling on, the event state change.
int apply_device_ws(bie_ctx* c, const double* sigma, double* yout, Workspace& ws) {
    return apply_impl(c, sigma, yout, BIE_MIXED, ws);
}

int rhs_device(bie_ctx* c, double* b) {
    int bs = 256, gs = (c->N + bs - 1) / bs;
    k_rhs<<<gs, bs, 0, c->stream>>>(c->nx, c->ny, c->node_cell, c->cells, c->N, reinterpret_cast<double2*>(b));
    BIE_LAUNCH(c, "k_rhs");
    return BIE_OK;
}

// ---------------------------------------------------------------------------
// Rigid-body velocities at the centroids and mu_eff.
// u(x^c) = sum_images sum_j G(x^c, y_j + s) q_j + sum_p G(x^c, y_p) xi_p
//          - sum_p G(C, y_p) xi_p;  curl by the closed form of the Stokeslet.
// Block (b, s): body b's centroid against source split s of its cell; split 0
// also adds the proxy terms.  vpart[(b * splits + s) * 3 + c].
// ---------------------------------------------------------------------------
// With the doubled-cell periodizer (imc non-null) each source node has its
// four images instead of the 3 x 3.
__global__ void __launch_bounds__(256)
k_velocities(const Src64* __restrict__ src, const double* __restrict__ body, const int* __restrict__ body_cell,
             const Cell* __restrict__ cells, const double* __restrict__ ypall, const double* __restrict__ xiall,
             int M, double* __restrict__ vpart, const int* __restrict__ imc) {
    __shared__ double red[33];
    const int b = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y;
    const int cidx = body_cell[b];
    const Cell& cl = cells[cidx];
    const double X = body[8 * b + 2], Y = body[8 * b + 3];
    double ux = 0, uy = 0, cu = 0;
    const int per = (cl.n_nodes + nsp - 1) / nsp;
    const int j0 = cl.node_off + sp * per, j1 = min(cl.node_off + cl.n_nodes, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        Src64 q = src[j];
        const int code = imc ? imc[j] : 0;
        for (int kk = 0; kk < (imc ? 4 : 9); ++kk) {
            const int k = imc ? img_shift(code, kk) : kk;
            double rx = X - (q.x + cl.sx[k]), ry = Y - (q.y + cl.sy[k]);
            double r2 = rx * rx + ry * ry;
            double rq = (rx * q.z + ry * q.w) / r2;
            double l = -0.5 * log(r2);
            ux += l * q.z + rx * rq;
            uy += l * q.w + ry * rq;
            cu += (ry * q.z - rx * q.w) / r2;
        }
    }
    if (sp == 0) {
        const double* yp = ypall + (size_t)cidx * 2 * M;
        const double* xi = xiall + (size_t)cidx * 2 * M;
        for (int p = threadIdx.x; p < M; p += blockDim.x) {
            double fx = xi[p], fy = xi[M + p];
            double rx = X - yp[2 * p], ry = Y - yp[2 * p + 1];
            double r2 = rx * rx + ry * ry;
            double rq = (rx * fx + ry * fy) / r2;
            double l = -0.5 * log(r2);
            ux += l * fx + rx * rq;
            uy += l * fy + ry * rq;
            cu += (ry * fx - rx * fy) / r2;
            rx = cl.C[0] - yp[2 * p];
            ry = cl.C[1] - yp[2 * p + 1];
            r2 = rx * rx + ry * ry;
            rq = (rx * fx + ry * fy) / r2;
            l = -0.5 * log(r2);
            ux -= l * fx + rx * rq;
            uy -= l * fy + ry * rq;
        }
    }
    ux = block_sum_d(ux, red);
    uy = block_sum_d(uy, red);
    cu = block_sum_d(cu, red);
    if (threadIdx.x == 0) {
        double* o = vpart + ((size_t)b * nsp + sp) * 3;
        o[0] = ux;
        o[1] = uy;
        o[2] = cu;
    }
}

__global__ void k_velocities_fin(const double* __restrict__ vpart, int nb, int nsp, const double* __restrict__ body,
                                 const int* __restrict__ body_cell, const Cell* __restrict__ cells,
                                 double* __restrict__ v, double* __restrict__ om) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Cell& cl = cells[body_cell[b]];
    double ux = 0, uy = 0, cu = 0;
    for (int s = 0; s < nsp; ++s) {
        const double* o = vpart + ((size_t)b * nsp + s) * 3;
        ux += o[0];
        uy += o[1];
        cu += o[2];
    }
    const double c4 = 1.0 / (4.0 * kPi * cl.mu);
    v[2 * b] = ux * c4 + cl.gamma * body[8 * b + 3];
    v[2 * b + 1] = uy * c4;
    om[b] = 0.5 * (cu / (2.0 * kPi * cl.mu) - cl.gamma);
}

// mu_eff per cell (one CTA per cell): the particle-stress average
__global__ void k_mu_eff(const double2* __restrict__ sigma, const double* __restrict__ y,
                         const double* __restrict__ w, const int* __restrict__ owner,
                         const double* __restrict__ body, const Cell* __restrict__ cells, double* __restrict__ out) {
    __shared__ double red[33];
    const Cell& cl = cells[blockIdx.x];
    double s = 0;
    for (int i = cl.node_off + threadIdx.x; i < cl.node_off + cl.n_nodes; i += blockDim.x)
        s += sigma[i].x * (y[i] - body[8 * owner[i] + 3]) * w[i];
    s = block_sum_d(s, red);
    const double area = fabs(cl.e1[0] * cl.e2[1] - cl.e1[1] * cl.e2[0]);
    if (threadIdx.x == 0) out[blockIdx.x] = cl.mu - s / (cl.gamma * area);
}

// The double-precision per-node sources, body moments and proxy strengths of
// sigma in the workspace (Sec. 6.2 steps 1-3 without the near sum); skipped
// when the workspace already holds them (reuse_ws).
int fp64_moments_and_xi(bie_ctx* c, const double* sigma, bool reuse_ws) {
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    if (!(reuse_ws && c->ws_x == sigma)) {
        if (c->utilde)
            k_pack_moments_u<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->body_cell, c->cells,
                                                           c->imc, nullptr, nullptr, c->ws.src64, nullptr, nullptr,
                                                           c->ws.bodyF);
        else
            k_pack_moments<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->body_cell, c->cells,
                                                         nullptr, c->ws.src64, nullptr, c->ws.bodyF);
        BIE_LAUNCH(c, "k_pack_moments");
        if (c->utilde)
            k_disc<false, true><<<dim3(2 * c->m, kDiscSplits, c->ncell), 256, 0, c->stream>>>(
                c->ws.src64, nullptr, c->cells, c->m, c->wall, c->ws.bodyF, c->ws.gpart, c->ws.dticket, c->ws.gt,
                c->imc);
        else
            k_disc<false, false><<<dim3(2 * c->m, kDiscSplits, c->ncell), 256, 0, c->stream>>>(
                c->ws.src64, nullptr, c->cells, c->m, c->wall, c->ws.bodyF, c->ws.gpart, c->ws.dticket, c->ws.gt,
                nullptr);
        BIE_LAUNCH(c, "k_disc");
        k_xi<<<dim3(2 * c->M, c->ncell), 32, 0, c->stream>>>(c->ws.gt, c->m, c->M, c->cells, c->P, c->ws.xi,
                                                               c->ws.xif);
        BIE_LAUNCH(c, "k_xi");
    }
    return BIE_OK;
}

int velocities_device(bie_ctx* c, const double* sigma, double* v, double* omega, double* mu_eff, bool reuse_ws) {
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    // reuse_ws: the time step calls this right after a solve whose last
    // (FP64-class) residual application was of this density over every
    // cell, so its sources, body moments and proxy strengths are reused
    if (int rc = fp64_moments_and_xi(c, sigma, reuse_ws)) return rc;
    if (v || omega) {
        k_velocities<<<dim3(c->nb, kVelSplits), 256, 0, c->stream>>>(c->ws.src64, c->body, c->body_cell, c->cells,
                                                                     c->yp, c->ws.xi, c->M, c->ws.vpart,
                                                                     c->utilde ? c->imc : nullptr);
        BIE_LAUNCH(c, "k_velocities");
        k_velocities_fin<<<(c->nb + 127) / 128, 128, 0, c->stream>>>(c->ws.vpart, c->nb, kVelSplits, c->body,
                                                                     c->body_cell, c->cells, v, omega);
        BIE_LAUNCH(c, "k_velocities_fin");
    }
    if (mu_eff) {
        k_mu_eff<<<c->ncell, 256, 0, c->stream>>>(sg, c->y, c->w, c->owner, c->body, c->cells, mu_eff);
        BIE_LAUNCH(c, "k_mu_eff");
    }
    return BIE_OK;
}

}  // namespace bie
