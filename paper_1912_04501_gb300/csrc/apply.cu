// The operator application y = A sigma (Eq. BIEdiscretized + L + pressure fix)
// and the velocity / effective-viscosity extraction.
//
// Launch sequence of one application (all on the context stream):
//   k_pack          q = sigma w; single- or double-precision source records
//   k_body_moments  F_b = sum q, tau_b = sum (x - x^c)^perp . q  (one CTA per body)
//   k_near32/64     3x3 near image sum of G^t at every node (Sec. 6.2 step 1),
//                   split over source chunks -> partial sums
//   k_disc          wall discrepancy of the near sum with the far-image
//                   cancellation (Sec. 6.2 step 2), split over source chunks
//   k_xi            g~ = g0 - g, xi = P g~ (Sec. 6.2 step 3)
//   k_correct       T = sum of partials + on-curve diagonal + proxy traction (step 4)
//   k_finish        alpha = -T_0 . n_0;  y = sigma/2 + T + alpha n + L sigma
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

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// ---------------------------------------------------------------------------
__global__ void k_pack(const double2* __restrict__ sigma, const double* __restrict__ x,
                       const double* __restrict__ y, const double* __restrict__ w, int N, double Cx,
                       double Cy, float4* __restrict__ src32, Src64* __restrict__ src64) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 s = sigma[i];
    double wi = w[i];
    double qx = s.x * wi, qy = s.y * wi;
    if (src32) src32[i] = make_float4((float)(x[i] - Cx), (float)(y[i] - Cy), (float)qx, (float)qy);
    if (src64) src64[i] = Src64{x[i], y[i], qx, qy};
}

__global__ void k_body_moments(const double2* __restrict__ sigma, const double* __restrict__ x,
                               const double* __restrict__ y, const double* __restrict__ w,
                               const double* __restrict__ body, double* __restrict__ bodyF) {
    __shared__ double red[33];
    int b = blockIdx.x;
    const double* bd = body + 8 * b;
    double xc = bd[2], yc = bd[3];
    int n = (int)bd[5], off = (int)bd[6];
    double fx = 0, fy = 0, tq = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        int i = off + k;
        double2 s = sigma[i];
        double qx = s.x * w[i], qy = s.y * w[i];
        fx += qx;
        fy += qy;
        tq += -(y[i] - yc) * qx + (x[i] - xc) * qy;
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

struct Shifts9 {
    float x[9], y[9];
};
struct Shifts9d {
    double x[9], y[9];
};

// ---------------------------------------------------------------------------
// Near image sum, single precision.  Block: kNearThreads threads, each owning
// TPT targets; grid.x over target tiles, grid.y over source chunks.  The 9
// image shifts are applied to the target (x_t - s) so every staged source is
// reused by 9 * TPT pair evaluations.  Per pair: 13 FP32 instructions and one
// MUFU reciprocal.  The zero-distance self pair is absorbed by a 1e-30 floor
// on r^2 (its r.n and r.q are exactly zero, so it contributes 0).
// ---------------------------------------------------------------------------
template <int TPT, bool COMP>
__global__ void __launch_bounds__(kNearThreads)
k_near32(const float4* __restrict__ tgt, const float4* __restrict__ src, int N, int chunk, Shifts9 sh,
         float2* __restrict__ part) {
    __shared__ float4 s_src[kNearTile];
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    float px[TPT][9], py[TPT][9], nxv[TPT], nyv[TPT];
    float ax[TPT][3], ay[TPT][3];
    // COMP: each source tile's sum is folded into a TwoSum-compensated pair
    // (hi, lo), so that splits with very many sources keep single-precision
    // accuracy relative to the sum instead of losing it to rounding growth.
    float hx[TPT], lx[TPT], hy[TPT], ly[TPT];
    int tbase = blockIdx.x * (kNearThreads * TPT) + threadIdx.x;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        int i = tbase + t * kNearThreads;
        float4 tv = i < N ? tgt[i] : make_float4(1e4f, 1e4f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            px[t][k] = tv.x - sh.x[k];
            py[t][k] = tv.y - sh.y[k];
        }
        nxv[t] = tv.z;
        nyv[t] = tv.w;
#pragma unroll
        for (int r = 0; r < 3; ++r) ax[t][r] = ay[t][r] = 0.f;
        hx[t] = lx[t] = hy[t] = ly[t] = 0.f;
    }
    for (int jt = j0; jt < j1; jt += kNearTile) {
        int cnt = min(kNearTile, j1 - jt);
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
                    float dx = px[t][im] - s.x;
                    float dy = py[t][im] - s.y;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, 1e-30f));
                    float rn = fmaf(dy, nyv[t], dx * nxv[t]);
                    float rq = fmaf(dy, s.w, dx * s.z);
                    float inv = rcp_approx(r2);
                    float cc = (rn * inv) * (rq * inv);
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
        if (i < N) {
            if constexpr (COMP)
                part[(size_t)blockIdx.y * N + i] = make_float2(c * (hx[t] + lx[t]), c * (hy[t] + ly[t]));
            else
                part[(size_t)blockIdx.y * N + i] =
                    make_float2(c * (ax[t][0] + ax[t][1] + ax[t][2]), c * (ay[t][0] + ay[t][1] + ay[t][2]));
        }
    }
}

// Near image sum, double precision (one target per thread).  Same structure;
// the self pair is absorbed by a 1e-300 floor on r^2.
__global__ void __launch_bounds__(kNearThreads)
k_near64(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
         const double* __restrict__ ny, const Src64* __restrict__ src, int N, int chunk, Shifts9d sh,
         double2* __restrict__ part) {
    __shared__ Src64 s_src[kNearTile];
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    int i = blockIdx.x * kNearThreads + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < N) {
        tx = x[i];
        ty = y[i];
        tnx = nx[i];
        tny = ny[i];
    }
    double px[9], py[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        px[k] = tx - sh.x[k];
        py[k] = ty - sh.y[k];
    }
    double ax[3] = {0, 0, 0}, ay[3] = {0, 0, 0};
    for (int jt = j0; jt < j1; jt += kNearTile) {
        int cnt = min(kNearTile, j1 - jt);
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
    if (i < N) {
        const double c = -1.0 / kPi;
        part[(size_t)blockIdx.y * N + i] = make_double2(c * (ax[0] + ax[1] + ax[2]), c * (ay[0] + ay[1] + ay[2]));
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
// dropped lo*lo cross terms stay at 2^-48; the accumulator keeps its TwoSum
// error in a float.  About 140 FP32 instructions per pair; each term is
// accurate to ~1e-14 of the kernel's scale |q| / |r| at any distance (the
// inputs carry 48 of double's 53 bits).
// ---------------------------------------------------------------------------
struct __align__(16) SrcDF {
    float xh, xl, yh, yl, qxh, qxl, qyh, qyl;
};

__device__ __forceinline__ void split_df(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// h + l -> normalised (|l| <= ulp(h) / 2), valid when |h| >= |l|
__device__ __forceinline__ void fast2(float& h, float& l) {
    float s = h + l;
    l = l - (s - h);
    h = s;
}

// (ph + pl) - (sh + sl), exact to ~2^-48 relative to the difference itself
__device__ __forceinline__ void df_diff(float ph, float pl, float sh, float sl, float& h, float& l) {
    float s1, e1, s2, e2, e3;
    two_sum(ph, -sh, s1, e1);
    two_sum(pl, -sl, s2, e2);
    two_sum(s1, s2, h, e3);
    l = (e1 + e2) + e3;
    fast2(h, l);
}

// (ah + al) * (bh + bl) -> (ph, pl), pl not renormalised
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    ph = ah * bh;
    pl = fmaf(ah, bh, -ph);
    pl = fmaf(ah, bl, fmaf(al, bh, pl));
}

__global__ void k_pack_df(const double2* __restrict__ sigma, const double* __restrict__ x,
                          const double* __restrict__ y, const double* __restrict__ w, int N, double Cx, double Cy,
                          SrcDF* __restrict__ src) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 s = sigma[i];
    double wi = w[i];
    SrcDF r;
    split_df(x[i] - Cx, r.xh, r.xl);
    split_df(y[i] - Cy, r.yh, r.yl);
    split_df(s.x * wi, r.qxh, r.qxl);
    split_df(s.y * wi, r.qyh, r.qyl);
    src[i] = r;
}

__global__ void __launch_bounds__(kNearThreads, 4)
k_near_df(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
          const double* __restrict__ ny, const SrcDF* __restrict__ src, int N, int chunk, Shifts9d sh, double Cx,
          double Cy, double2* __restrict__ part) {
    __shared__ SrcDF s_src[kNearTile];
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    const int i = blockIdx.x * kNearThreads + threadIdx.x;
    double tx = 1e4, ty = 1e4, tnx = 0, tny = 0;
    if (i < N) {
        tx = x[i] - Cx;
        ty = y[i] - Cy;
        tnx = nx[i];
        tny = ny[i];
    }
    float pxh[9], pxl[9], pyh[9], pyl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        split_df(tx - sh.x[k], pxh[k], pxl[k]);
        split_df(ty - sh.y[k], pyh[k], pyl[k]);
    }
    float nxh, nxl, nyh, nyl;
    split_df(tnx, nxh, nxl);
    split_df(tny, nyh, nyl);
    // per tile: hi sums by TwoSum, their errors in a float; folded into double
    // accumulators after every tile so that neither grows with the source count
    double dxs = 0, dys = 0;
    for (int jt = j0; jt < j1; jt += kNearTile) {
        int cnt = min(kNearTile, j1 - jt);
        float axh = 0, axe = 0, ayh = 0, aye = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += kNearThreads) s_src[k] = src[jt + k];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const SrcDF q = s_src[k];
#pragma unroll
            for (int im = 0; im < 9; ++im) {
                float rxh, rxl, ryh, ryl, e;
                df_diff(pxh[im], pxl[im], q.xh, q.xl, rxh, rxl);
                df_diff(pyh[im], pyl[im], q.yh, q.yl, ryh, ryl);
                // r^2 (the 1e-30 floor absorbs the zero-distance self pair)
                float a, ea, b, eb, r2h, r2l;
                a = rxh * rxh;
                ea = fmaf(rxh, rxh, -a);
                ea = fmaf(rxh, rxl + rxl, ea);
                b = ryh * ryh;
                eb = fmaf(ryh, ryh, -b);
                eb = fmaf(ryh, ryl + ryl, eb);
                two_sum(a, b, r2h, e);
                r2l = e + ea + eb;
                r2h += 1e-30f;
                // 1 / r^2
                const float ih = rcp_approx(r2h);
                float res = fmaf(-r2h, ih, 1.0f);
                res = fmaf(-r2l, ih, res);
                const float il = ih * res;
                // r . n and r . q
                float p1, e1, p2, e2, rnh, rnl, rqh, rql;
                df_mul(rxh, rxl, nxh, nxl, p1, e1);
                df_mul(ryh, ryl, nyh, nyl, p2, e2);
                two_sum(p1, p2, rnh, e);
                rnl = e + e1 + e2;
                fast2(rnh, rnl);  // r.n may cancel: renormalise before multiplying
                df_mul(rxh, rxl, q.qxh, q.qxl, p1, e1);
                df_mul(ryh, ryl, q.qyh, q.qyl, p2, e2);
                two_sum(p1, p2, rqh, e);
                rql = e + e1 + e2;
                fast2(rqh, rql);
                // c = (r.n / r^2) (r.q / r^2), term = c r
                float uh, ul, vh, vl, ch, cl, th, tl;
                df_mul(rnh, rnl, ih, il, uh, ul);
                df_mul(rqh, rql, ih, il, vh, vl);
                df_mul(uh, ul, vh, vl, ch, cl);
                df_mul(ch, cl, rxh, rxl, th, tl);
                two_sum(axh, th, axh, e);
                axe += e + tl;
                df_mul(ch, cl, ryh, ryl, th, tl);
                two_sum(ayh, th, ayh, e);
                aye += e + tl;
            }
        }
        dxs += (double)axh + (double)axe;
        dys += (double)ayh + (double)aye;
    }
    if (i < N) {
        const double c = -1.0 / kPi;
        part[(size_t)blockIdx.y * N + i] = make_double2(c * dxs, c * dys);
    }
}

// ---------------------------------------------------------------------------
// Wall table (per geometry): for each collocation point (L points, then D
// points) the point minus each of its six far-image shifts, and the wall
// normal used for the traction.
__global__ void k_wall_table(int m, const double* __restrict__ gl_s, double e1x, double e1y, double e2x,
                             double e2y, double Cx, double Cy, double* __restrict__ wall) {
    int wp = blockIdx.x * blockDim.x + threadIdx.x;
    if (wp >= 2 * m) return;
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
    double* o = wall + 16 * wp;
    for (int k = -1; k <= 1; ++k) {
        o[2 * (k + 1)] = X - (-2.0 * ax + k * bx);
        o[2 * (k + 1) + 1] = Y - (-2.0 * ay + k * by);
        o[2 * (k + 4)] = X - (ax + k * bx);
        o[2 * (k + 4) + 1] = Y - (ay + k * by);
    }
    o[12] = isL ? nl[0] : nd[0];
    o[13] = isL ? nl[1] : nd[1];
}

int build_wall_table(bie_ctx* c, const double* e2, double* wall, cudaStream_t st) {
    k_wall_table<<<(2 * c->m + 63) / 64, 64, 0, st>>>(c->m, c->gl_s, c->e1[0], c->e1[1], e2[0], e2[1], c->C[0],
                                                      c->C[1], wall);
    BIE_LAUNCH(c, "k_wall_table");
    return BIE_OK;
}

// Wall discrepancy (Sec. 6.2 step 2).  For a collocation point x on L,
//   S_near(x + e1) - S_near(x) = sum_n sum_j [K(x, y_j - 2 e1 + n e2) - K(x, y_j + e1 + n e2)] q_j
// and on D with the roles of e1, e2 exchanged; K is the velocity kernel G or
// the traction kernel G^t with the wall normal.  Block (wp, s): wall point
// wp in [0, 2m) (L points, then D points) and source split s of kDiscSplits;
// its threads stride over the split's sources and the block reduces
// (u_x, u_y, t_x, t_y) into gpart[(s * 2m + wp) * 4 + comp].
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fast_log(float x) { return __logf(x); }
__device__ __forceinline__ double fast_log(double x) { return log(x); }
__device__ __forceinline__ float fast_rcp(float x) { return rcp_approx(x); }
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

template <typename Real>
__global__ void __launch_bounds__(256)
k_disc(const Src64* __restrict__ src, int N, int m, const double* __restrict__ wall, double mu,
       double* __restrict__ gpart) {
    __shared__ double red[4][33];
    const int wp = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y;
    // per-geometry table: collocation point minus each of the six far-image
    // shifts (plus images -2a + kb, then minus images a + kb), and the normal
    const double* wt = wall + 16 * wp;
    Real ox[6], oy[6];
#pragma unroll
    for (int im = 0; im < 6; ++im) {
        ox[im] = (Real)wt[2 * im];
        oy[im] = (Real)wt[2 * im + 1];
    }
    const Real n0 = (Real)wt[12], n1 = (Real)wt[13];
    Real ux = 0, uy = 0, tx = 0, ty = 0;
    const int per = (N + nsp - 1) / nsp;
    const int j0 = sp * per, j1 = min(N, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const Src64 q = src[j];
        const Real qx = (Real)q.z, qy = (Real)q.w, sx = (Real)q.x, sy = (Real)q.y;
#pragma unroll
        for (int im = 0; im < 6; ++im) {
            const Real rx = ox[im] - sx, ry = oy[im] - sy;
            const Real r2 = rx * rx + ry * ry;
            const Real inv = fast_rcp(r2);
            const Real rq = rx * qx + ry * qy;
            const Real l = (Real)(-0.5) * fast_log(r2);
            const Real a = rq * inv;
            const Real vx = l * qx + rx * a, vy = l * qy + ry * a;
            const Real cc = (rx * n0 + ry * n1) * a * inv;
            if (im < 3) {
                ux += vx; uy += vy; tx += cc * rx; ty += cc * ry;
            } else {
                ux -= vx; uy -= vy; tx -= cc * rx; ty -= cc * ry;
            }
        }
    }
    double v[4] = {(double)ux, (double)uy, (double)tx, (double)ty};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double t = v[c];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[c][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0;
        for (int k = 0; k < nw; ++k) t += red[threadIdx.x][k];
        const double scale = threadIdx.x < 2 ? 1.0 / (4.0 * kPi * mu) : -1.0 / kPi;
        gpart[((size_t)sp * 2 * m + wp) * 4 + threadIdx.x] = t * scale;
    }
}

// g~ and xi = P g~ (Sec. 6.2 step 3).  One warp-sized CTA per row r of P (2M
// CTAs): GB300's FP64 pipe is narrow, so the compensated products are spread
// over as many SMs as there are rows.  Every CTA rebuilds g~ from the kDiscSplits
// partials of the discrepancy kernel (fixed order: deterministic) and then
// computes xi_r with a compensated dot product (Ogita, Rump & Oishi's Dot2:
// FMA-exact products, error-free sums; P has entries up to ~1/lam, so a plain
// double-precision product would add relative noise ~1e-11 to the correction
// and put a floor under the GMRES residual).
__global__ void __launch_bounds__(32)
k_xi(const double* __restrict__ gpart, int nblk, int m, int M, const double* __restrict__ bodyF, int nb,
     double l1, double l2, const double* __restrict__ P, double* __restrict__ xi) {
    extern __shared__ double d[];  // 8m: g~
    const int lane = threadIdx.x, r = blockIdx.x;
    const int nv = 8 * m;
    double fx = 0, fy = 0;
    for (int b = lane; b < nb; b += 32) {
        fx += bodyF[3 * b];
        fy += bodyF[3 * b + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
    }
    for (int wp = lane; wp < 2 * m; wp += 32) {
        double g[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double a = 0;
            for (int b = 0; b < nblk; ++b) a += gpart[(size_t)b * nv + 4 * wp + c];
            g[c] = a;
        }
        if (wp < m) {  // L: rows of blocks 1 (velocity) and 2 (traction)
            const int l = wp;
            d[l] = -g[0];
            d[m + l] = -g[1];
            d[2 * m + l] = fx / (2.0 * l2) - g[2];
            d[3 * m + l] = fy / (2.0 * l2) - g[3];
        } else {  // D: blocks 3 and 4
            const int l = wp - m;
            d[4 * m + l] = -g[0];
            d[5 * m + l] = -g[1];
            d[6 * m + l] = fx / (2.0 * l1) - g[2];
            d[7 * m + l] = fy / (2.0 * l1) - g[3];
        }
    }
    __syncwarp();
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
    if (lane == 0) xi[r] = s + e;
}

// T = near partials + on-curve diagonal -(kappa/2pi) tau (tau . q) + proxy
// traction.  ProxyReal = float on the single-precision path (rcp.approx, the
// inner-solve operator), double on the FP64 path.
template <typename PartT, typename ProxyReal>
__global__ void __launch_bounds__(256)
k_correct(const PartT* __restrict__ part, int splits, int N, const double2* __restrict__ sigma,
          const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
          const double* __restrict__ ny, const double* __restrict__ w, const double* __restrict__ kap,
          const double* __restrict__ yp, const double* __restrict__ xi, int M, double Cx, double Cy,
          double2* __restrict__ T) {
    // kCorrLanes lanes per target: they split the near-sum partials and the
    // proxies, then combine with shuffles (fixed order: deterministic)
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) / kCorrLanes;
    const int sub = threadIdx.x % kCorrLanes;
    const int i = g < N ? g : N - 1;
    double tx = 0, ty = 0;
    for (int s = sub; s < splits; s += kCorrLanes) {
        PartT p = part[(size_t)s * N + i];
        tx += (double)p.x;
        ty += (double)p.y;
    }
    const double n0 = nx[i], n1 = ny[i];
    // proxies in cell-centred coordinates (exact in double, accurate in float)
    const ProxyReal X = (ProxyReal)(x[i] - Cx), Y = (ProxyReal)(y[i] - Cy);
    const ProxyReal m0 = (ProxyReal)n0, m1 = (ProxyReal)n1;
    ProxyReal cx = 0, cy = 0;
    for (int p = sub; p < M; p += kCorrLanes) {
        ProxyReal rx = X - (ProxyReal)(yp[2 * p] - Cx), ry = Y - (ProxyReal)(yp[2 * p + 1] - Cy);
        ProxyReal fx = (ProxyReal)xi[p], fy = (ProxyReal)xi[M + p];
        ProxyReal r2 = rx * rx + ry * ry;
        ProxyReal inv;
        if constexpr (sizeof(ProxyReal) == 4) inv = rcp_approx(r2);
        else inv = (ProxyReal)1 / r2;
        ProxyReal cc = ((rx * m0 + ry * m1) * inv) * ((rx * fx + ry * fy) * inv);
        cx += cc * rx;
        cy += cc * ry;
    }
    tx += -(double)cx / kPi;
    ty += -(double)cy / kPi;
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

__global__ void k_finish(const double2* __restrict__ T, const double2* __restrict__ sigma, int N,
                         const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ nx, const double* __restrict__ ny,
                         const int* __restrict__ owner, const double* __restrict__ body,
                         const double* __restrict__ bodyF, double2* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 T0 = T[0];
    double alpha = -(T0.x * nx[0] + T0.y * ny[0]);
    int b = owner[i];
    double xc = body[8 * b + 2], yc = body[8 * b + 3];
    double Fx = bodyF[3 * b], Fy = bodyF[3 * b + 1], tq = bodyF[3 * b + 2];
    double2 Ti = T[i], s = sigma[i];
    double ox = 0.5 * s.x + Ti.x + alpha * nx[i] + Fx - (y[i] - yc) * tq;
    double oy = 0.5 * s.y + Ti.y + alpha * ny[i] + Fy + (x[i] - xc) * tq;
    out[i] = make_double2(ox, oy);
}

__global__ void k_rhs(const double* __restrict__ nx, const double* __restrict__ ny, int N, double mg,
                      double2* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) b[i] = make_double2(-mg * ny[i], -mg * nx[i]);
}

// ---------------------------------------------------------------------------
static void shifts(const bie_ctx* c, double* sx, double* sy, bool centred) {
    int k = 0;
    for (int n = -1; n <= 1; ++n)
        for (int mm = -1; mm <= 1; ++mm, ++k) {
            sx[k] = mm * c->e1[0] + n * c->e2[0];
            sy[k] = mm * c->e1[1] + n * c->e2[1];
        }
    (void)centred;
}

int apply_device(bie_ctx* c, const double* sigma, double* yout, int precision) {
    const int N = c->N;
    const int bs = 256, gs = (N + bs - 1) / bs;
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    bool f32 = precision == BIE_MIXED;
    bool df = precision == BIE_DF64;
    k_pack<<<gs, bs, 0, c->stream>>>(sg, c->x, c->y, c->w, N, c->C[0], c->C[1], f32 ? c->ws.src32 : nullptr,
                                     c->ws.src64);
    BIE_LAUNCH(c, "k_pack");
    if (df) {
        k_pack_df<<<gs, bs, 0, c->stream>>>(sg, c->x, c->y, c->w, N, c->C[0], c->C[1], (SrcDF*)c->ws.srcdf);
        BIE_LAUNCH(c, "k_pack_df");
    }
    k_body_moments<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->ws.bodyF);
    BIE_LAUNCH(c, "k_body_moments");
    double sx[9], sy[9];
    shifts(c, sx, sy, false);
    int splits;
    if (f32) {
        Shifts9 s9;
        for (int k = 0; k < 9; ++k) {
            s9.x[k] = (float)sx[k];
            s9.y[k] = (float)sy[k];
        }
        splits = c->near_splits32;
        int tiles = (N + kNearThreads * kNear32TPT - 1) / (kNearThreads * kNear32TPT);
        int chunk = (N + splits - 1) / splits;
        dim3 grid(tiles, splits);
        if (int rc = prof_begin(c, 0)) return rc;
        if (chunk > kNear32CompChunk)
            k_near32<kNear32TPT, true><<<grid, kNearThreads, 0, c->stream>>>(c->tgt32, c->ws.src32, N, chunk, s9,
                                                                             (float2*)c->ws.part);
        else
            k_near32<kNear32TPT, false><<<grid, kNearThreads, 0, c->stream>>>(c->tgt32, c->ws.src32, N, chunk, s9,
                                                                              (float2*)c->ws.part);
        BIE_LAUNCH(c, "k_near32");
        if (int rc = prof_end(c)) return rc;
    } else if (df) {
        Shifts9d s9;
        for (int k = 0; k < 9; ++k) {
            s9.x[k] = sx[k];
            s9.y[k] = sy[k];
        }
        splits = c->near_splitsdf;
        int tiles = (N + kNearThreads - 1) / kNearThreads;
        int chunk = (N + splits - 1) / splits;
        dim3 grid(tiles, splits);
        if (int rc = prof_begin(c, 2)) return rc;
        k_near_df<<<grid, kNearThreads, 0, c->stream>>>(c->x, c->y, c->nx, c->ny, (const SrcDF*)c->ws.srcdf, N, chunk,
                                                        s9, c->C[0], c->C[1], (double2*)c->ws.part);
        BIE_LAUNCH(c, "k_near_df");
        if (int rc = prof_end(c)) return rc;
    } else {
        Shifts9d s9;
        for (int k = 0; k < 9; ++k) {
            s9.x[k] = sx[k];
            s9.y[k] = sy[k];
        }
        splits = c->near_splits64;
        int tiles = (N + kNearThreads - 1) / kNearThreads;
        int chunk = (N + splits - 1) / splits;
        dim3 grid(tiles, splits);
        if (int rc = prof_begin(c, 1)) return rc;
        k_near64<<<grid, kNearThreads, 0, c->stream>>>(c->x, c->y, c->nx, c->ny, c->ws.src64, N, chunk, s9,
                                                       (double2*)c->ws.part);
        BIE_LAUNCH(c, "k_near64");
        if (int rc = prof_end(c)) return rc;
    }
    if (f32)
        k_disc<float><<<dim3(2 * c->m, kDiscSplits), 256, 0, c->stream>>>(c->ws.src64, N, c->m, c->wall, c->mu, c->ws.gpart);
    else
        k_disc<double><<<dim3(2 * c->m, kDiscSplits), 256, 0, c->stream>>>(c->ws.src64, N, c->m, c->wall, c->mu, c->ws.gpart);
    BIE_LAUNCH(c, "k_disc");
    double l1 = sqrt(c->e1[0] * c->e1[0] + c->e1[1] * c->e1[1]);
    double l2 = sqrt(c->e2[0] * c->e2[0] + c->e2[1] * c->e2[1]);
    k_xi<<<2 * c->M, 32, 8 * c->m * sizeof(double), c->stream>>>(c->ws.gpart, kDiscSplits, c->m, c->M, c->ws.bodyF,
                                                          c->nb, l1, l2, c->P, c->ws.xi);
    BIE_LAUNCH(c, "k_xi");
    double2* T = reinterpret_cast<double2*>(c->ws.T);
    const int gsc = (N * kCorrLanes + 255) / 256;
    if (f32)
        k_correct<float2, float><<<gsc, 256, 0, c->stream>>>((const float2*)c->ws.part, splits, N, sg, c->x, c->y,
                                                             c->nx, c->ny, c->w, c->kap, c->yp, c->ws.xi, c->M,
                                                             c->C[0], c->C[1], T);
    else
        k_correct<double2, double><<<gsc, 256, 0, c->stream>>>((const double2*)c->ws.part, splits, N, sg, c->x,
                                                               c->y, c->nx, c->ny, c->w, c->kap, c->yp, c->ws.xi,
                                                               c->M, c->C[0], c->C[1], T);
    BIE_LAUNCH(c, "k_correct");
    if (int rc = close_apply(c, sigma, c->ws.T)) return rc;
    k_finish<<<gs, bs, 0, c->stream>>>(T, sg, N, c->x, c->y, c->nx, c->ny, c->owner, c->body, c->ws.bodyF,
                                       reinterpret_cast<double2*>(yout));
    BIE_LAUNCH(c, "k_finish");
    return BIE_OK;
}

int rhs_device(bie_ctx* c, double* b) {
    int bs = 256, gs = (c->N + bs - 1) / bs;
    k_rhs<<<gs, bs, 0, c->stream>>>(c->nx, c->ny, c->N, c->mu * c->gamma, reinterpret_cast<double2*>(b));
    BIE_LAUNCH(c, "k_rhs");
    return BIE_OK;
}

// ---------------------------------------------------------------------------
// Rigid-body velocities at the centroids (one CTA per body) and mu_eff.
// u(x^c) = sum_images sum_j G(x^c, y_j + s) q_j + sum_p G(x^c, y_p) xi_p
//          - sum_p G(C, y_p) xi_p;  curl by the closed form of the Stokeslet.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_velocities(const Src64* __restrict__ src, int N, Shifts9d sh, const double* __restrict__ body,
             const double* __restrict__ yp, const double* __restrict__ xi, int M, double Cx, double Cy,
             double* __restrict__ vpart) {
    // block (b, s): body b's centroid against source split s of gridDim.y;
    // split 0 also adds the proxy terms.  vpart[(b * splits + s) * 3 + c].
    __shared__ double red[33];
    const int b = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y;
    const double X = body[8 * b + 2], Y = body[8 * b + 3];
    double ux = 0, uy = 0, cu = 0;
    const int per = (N + nsp - 1) / nsp;
    const int j0 = sp * per, j1 = min(N, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        Src64 q = src[j];
        for (int k = 0; k < 9; ++k) {
            double rx = X - (q.x + sh.x[k]), ry = Y - (q.y + sh.y[k]);
            double r2 = rx * rx + ry * ry;
            double rq = (rx * q.z + ry * q.w) / r2;
            double l = -0.5 * log(r2);
            ux += l * q.z + rx * rq;
            uy += l * q.w + ry * rq;
            cu += (ry * q.z - rx * q.w) / r2;
        }
    }
    if (sp == 0) {
        for (int p = threadIdx.x; p < M; p += blockDim.x) {
            double fx = xi[p], fy = xi[M + p];
            double rx = X - yp[2 * p], ry = Y - yp[2 * p + 1];
            double r2 = rx * rx + ry * ry;
            double rq = (rx * fx + ry * fy) / r2;
            double l = -0.5 * log(r2);
            ux += l * fx + rx * rq;
            uy += l * fy + ry * rq;
            cu += (ry * fx - rx * fy) / r2;
            rx = Cx - yp[2 * p];
            ry = Cy - yp[2 * p + 1];
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
                                 double mu, double gamma, double* __restrict__ v, double* __restrict__ om) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double ux = 0, uy = 0, cu = 0;
    for (int s = 0; s < nsp; ++s) {
        const double* o = vpart + ((size_t)b * nsp + s) * 3;
        ux += o[0];
        uy += o[1];
        cu += o[2];
    }
    const double c4 = 1.0 / (4.0 * kPi * mu);
    v[2 * b] = ux * c4 + gamma * body[8 * b + 3];
    v[2 * b + 1] = uy * c4;
    om[b] = 0.5 * (cu / (2.0 * kPi * mu) - gamma);
}

__global__ void k_mu_eff(const double2* __restrict__ sigma, const double* __restrict__ y,
                         const double* __restrict__ w, const int* __restrict__ owner,
                         const double* __restrict__ body, int N, double mu, double gamma, double area,
                         double* __restrict__ out) {
    __shared__ double red[33];
    double s = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += sigma[i].x * (y[i] - body[8 * owner[i] + 3]) * w[i];
    s = block_sum_d(s, red);
    if (threadIdx.x == 0) *out = mu - s / (gamma * area);
}

int velocities_device(bie_ctx* c, const double* sigma, double* v, double* omega, double* mu_eff) {
    const int N = c->N;
    const int bs = 256, gs = (N + bs - 1) / bs;
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    k_pack<<<gs, bs, 0, c->stream>>>(sg, c->x, c->y, c->w, N, c->C[0], c->C[1], nullptr, c->ws.src64);
    BIE_LAUNCH(c, "k_pack");
    k_body_moments<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, c->ws.bodyF);
    BIE_LAUNCH(c, "k_body_moments");
    k_disc<double><<<dim3(2 * c->m, kDiscSplits), 256, 0, c->stream>>>(c->ws.src64, N, c->m, c->wall, c->mu, c->ws.gpart);
    BIE_LAUNCH(c, "k_disc");
    double l1 = sqrt(c->e1[0] * c->e1[0] + c->e1[1] * c->e1[1]);
    double l2 = sqrt(c->e2[0] * c->e2[0] + c->e2[1] * c->e2[1]);
    k_xi<<<2 * c->M, 32, 8 * c->m * sizeof(double), c->stream>>>(c->ws.gpart, kDiscSplits, c->m, c->M, c->ws.bodyF,
                                                          c->nb, l1, l2, c->P, c->ws.xi);
    BIE_LAUNCH(c, "k_xi");
    double sx[9], sy[9];
    shifts(c, sx, sy, false);
    Shifts9d s9;
    for (int k = 0; k < 9; ++k) {
        s9.x[k] = sx[k];
        s9.y[k] = sy[k];
    }
    if (v || omega) {
        k_velocities<<<dim3(c->nb, kVelSplits), 256, 0, c->stream>>>(c->ws.src64, N, s9, c->body, c->yp, c->ws.xi,
                                                                     c->M, c->C[0], c->C[1], c->ws.vpart);
        BIE_LAUNCH(c, "k_velocities");
        k_velocities_fin<<<(c->nb + 127) / 128, 128, 0, c->stream>>>(c->ws.vpart, c->nb, kVelSplits, c->body, c->mu,
                                                                     c->gamma, v, omega);
        BIE_LAUNCH(c, "k_velocities_fin");
    }
    if (mu_eff) {
        double area = fabs(c->e1[0] * c->e2[1] - c->e1[1] * c->e2[0]);
        k_mu_eff<<<1, 1024, 0, c->stream>>>(sg, c->y, c->w, c->owner, c->body, N, c->mu, c->gamma, area, mu_eff);
        BIE_LAUNCH(c, "k_mu_eff");
    }
    return BIE_OK;
}

}  // namespace bie

namespace bie {

// The single-precision-pair operator application with every per-call buffer
// taken from `ws` (used by the allocation-free entry point, whose buffers
// live in a static device array).  The kernels and their order are those of
// apply_device; the context is only read.
int apply_device_ws(bie_ctx* c, const double* sigma, double* yout, Workspace& ws) {
    const int N = c->N;
    const int bs = 256, gs = (N + bs - 1) / bs;
    const double2* sg = reinterpret_cast<const double2*>(sigma);
    k_pack<<<gs, bs, 0, c->stream>>>(sg, c->x, c->y, c->w, N, c->C[0], c->C[1], ws.src32, ws.src64);
    BIE_LAUNCH(c, "k_pack");
    k_body_moments<<<c->nb, 256, 0, c->stream>>>(sg, c->x, c->y, c->w, c->body, ws.bodyF);
    BIE_LAUNCH(c, "k_body_moments");
    double sx[9], sy[9];
    shifts(c, sx, sy, false);
    Shifts9 s9;
    for (int k = 0; k < 9; ++k) {
        s9.x[k] = (float)sx[k];
        s9.y[k] = (float)sy[k];
    }
    const int splits = c->near_splits32;
    const int tiles = (N + kNearThreads * kNear32TPT - 1) / (kNearThreads * kNear32TPT);
    const int chunk = (N + splits - 1) / splits;
    if (chunk > kNear32CompChunk)
        k_near32<kNear32TPT, true><<<dim3(tiles, splits), kNearThreads, 0, c->stream>>>(c->tgt32, ws.src32, N, chunk,
                                                                                       s9, (float2*)ws.part);
    else
        k_near32<kNear32TPT, false><<<dim3(tiles, splits), kNearThreads, 0, c->stream>>>(c->tgt32, ws.src32, N,
                                                                                        chunk, s9, (float2*)ws.part);
    BIE_LAUNCH(c, "k_near32");
    k_disc<float><<<dim3(2 * c->m, kDiscSplits), 256, 0, c->stream>>>(ws.src64, N, c->m, c->wall, c->mu, ws.gpart);
    BIE_LAUNCH(c, "k_disc");
    const double l1 = sqrt(c->e1[0] * c->e1[0] + c->e1[1] * c->e1[1]);
    const double l2 = sqrt(c->e2[0] * c->e2[0] + c->e2[1] * c->e2[1]);
    k_xi<<<2 * c->M, 32, 8 * c->m * sizeof(double), c->stream>>>(ws.gpart, kDiscSplits, c->m, c->M, ws.bodyF, c->nb, l1,
                                                          l2, c->P, ws.xi);
    BIE_LAUNCH(c, "k_xi");
    double2* T = reinterpret_cast<double2*>(ws.T);
    k_correct<float2, float><<<(N * kCorrLanes + 255) / 256, 256, 0, c->stream>>>((const float2*)ws.part, splits, N, sg, c->x,
                                                                  c->y, c->nx, c->ny, c->w, c->kap, c->yp, ws.xi,
                                                                  c->M, c->C[0], c->C[1], T);
    BIE_LAUNCH(c, "k_correct");
    if (int rc = close_apply(c, sigma, ws.T)) return rc;
    k_finish<<<gs, bs, 0, c->stream>>>(T, sg, N, c->x, c->y, c->nx, c->ny, c->owner, c->body, ws.bodyF,
                                       reinterpret_cast<double2*>(yout));
    BIE_LAUNCH(c, "k_finish");
    return BIE_OK;
}

}  // namespace bie
