// Close-evaluation correction (Sec. 6.3 and its remark on the two-phase
// solver): a sparse set of 2 x 2N_b blocks, built once per geometry, applied
// in every operator application.
//
// For a target x_i (normal n_i) within close_factor * h_b of an image of body
// b (h_b = perimeter / N_b), the smooth N_b-point rule for
//     int_{Gamma_b + s} G^t(x_i, y; n_i) sigma(y) ds_y
// is replaced by the same integral of the trigonometric interpolant of the
// nodal density, evaluated by the trapezoidal rule on rho * N_b points of the
// exact ellipse, rho >= 2 the smallest power of two with
// rho - 1/2 >= 6.4 h_loc / d (d the distance to the curve and h_loc the local
// node spacing at the closest point, both found by Newton's method).  As a linear map of the nodal density this is
//     C_k = sum_f G^t(x_i, y_f + s; n_i) w_f D(t_f - t_k) - G^t(x_i, y_k + s; n_i) w_k,
// D the Dirichlet kernel of the N_b-point interpolant (Nyquist mode split),
//     D(tau) = sin(N_b tau / 2) cot(tau / 2) / N_b.
// G^t applied to q is c r (r . q) with c = -(r . n)/(pi r^4), so each C_k is
// a symmetric 2 x 2 matrix: three doubles (A, B, D) per node.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

// h_b and the bounding radius per body (body[8b+7] = h_b).
__global__ void k_body_h(const double* __restrict__ w, double* __restrict__ body) {
    __shared__ double red[33];
    int b = blockIdx.x;
    double* bd = body + 8 * b;
    int n = (int)bd[5], off = (int)bd[6];
    double s = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += w[off + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        bd[7] = t / n;
    }
}

// One thread per target: every (body, image) of the target's cell closer than
// close_factor * h_b goes to the target's slots in (body, image) order.  slot
// record: int4 (body, image, rho, 0).  Distances to the curve below gap_lim
// (other bodies and the target's own periodic images) lower *gap_min, the
// bit pattern of a non-negative double (such patterns order like integers).
// With the doubled-cell periodizer (imc non-null) a pair is valid only when
// the body image, seen from the target's translate inside U, is among the
// images of every node of the body (bimg); otherwise bit 1 of *gflag is set.
__global__ void k_close_detect(const double* __restrict__ x, const double* __restrict__ y,
                               const int* __restrict__ owner, const double* __restrict__ body,
                               const int* __restrict__ node_cell, const Cell* __restrict__ cells, int N,
                               double close_factor, double gap_lim, int kmax, int4* __restrict__ slots,
                               int* __restrict__ count, int* __restrict__ overflow,
                               unsigned long long* __restrict__ gap_min, int* __restrict__ rho_max,
                               float* __restrict__ dmin, float2* __restrict__ ddir, const int* __restrict__ imc,
                               const int4* __restrict__ bimg, int* __restrict__ gflag,
                               const double* __restrict__ bshape) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Cell& sh = cells[node_cell[i]];
    const int wi = imc ? img_wrap(imc[i]) : 4;  // the target's translate into U
    double X = x[i], Y = y[i];
    int own = owner[i];
    int c = 0;
    double dbest = INFINITY, dirx = 0, diry = 0;  // nearest other curve (or own periodic image)
    for (int b = sh.body_off; b < sh.body_off + sh.n_bodies; ++b) {
        const double* bd = body + 8 * b;
        double R = fmax(bd[0], bd[1]);
        double hb = bd[7];
        double zone = close_factor * hb;
        double lim = fmax(zone, gap_lim);
        int n = (int)bd[5], off = (int)bd[6];
        for (int im = 0; im < 9; ++im) {
            if (b == own && im == 4) continue;  // zero shift of the own body
            double cx = bd[2] + sh.sx[im], cy = bd[3] + sh.sy[im];
            double dc = sqrt((X - cx) * (X - cx) + (Y - cy) * (Y - cy));
            if (dc - R > lim) continue;
            double d2 = 1e300;
            int kbest = 0;
            for (int k = 0; k < n; ++k) {
                double dx = X - (x[off + k] + sh.sx[im]), dy = Y - (y[off + k] + sh.sy[im]);
                double e = dx * dx + dy * dy;
                if (e < d2) { d2 = e; kbest = k; }
            }
            if (sqrt(d2) >= lim) continue;
            // distance to the exact curve and local node spacing at the closest
            // point: Newton on (y(t) - x) . y'(t) = 0 from the nearest node
            double dcur, hloc;
            const double* shp = bshape + 4 * b;
            if (shp[0] == 1.0) {
                // star: Newton on g(t) = (p(t) - u) . p'(t), g' = |p'|^2 + (p - u) . p''
                double st, ct;
                sincos(bd[4], &st, &ct);
                const double px = X - cx, py = Y - cy;
                const double u = ct * px + st * py, v = -st * px + ct * py;
                const double dtm = 2.0 * kPi / n;
                double t = dtm * kbest, qx, qy, dqx, dqy, ddqx, ddqy;
                for (int it = 0; it < 8; ++it) {
                    star_curve(shp, t, qx, qy, dqx, dqy, ddqx, ddqy);
                    const double g = (qx - u) * dqx + (qy - v) * dqy;
                    const double gp = dqx * dqx + dqy * dqy + (qx - u) * ddqx + (qy - v) * ddqy;
                    const double step = gp > 0 ? g / gp : copysign(dtm, g);
                    t -= fmax(-dtm, fmin(dtm, step));
                }
                star_curve(shp, t, qx, qy, dqx, dqy, ddqx, ddqy);
                dcur = sqrt((qx - u) * (qx - u) + (qy - v) * (qy - v));
                hloc = 2.0 * kPi * sqrt(dqx * dqx + dqy * dqy) / n;
                if (dcur < dbest && dcur > 0) {
                    const double ex = (qx - u) / dcur, ey = (qy - v) / dcur;
                    dbest = dcur;
                    dirx = ct * ex - st * ey;
                    diry = st * ex + ct * ey;
                }
            } else {
                double a = bd[0], b2 = bd[1], st, ct;
                sincos(bd[4], &st, &ct);
                double px = X - cx, py = Y - cy;
                double u = ct * px + st * py, v = -st * px + ct * py;
                double dtm = 2.0 * kPi / n, t = dtm * kbest;
                for (int it = 0; it < 8; ++it) {
                    double sn, cs;
                    sincos(t, &sn, &cs);
                    double g = (b2 * b2 - a * a) * sn * cs + a * u * sn - b2 * v * cs;
                    double gp = (b2 * b2 - a * a) * (cs * cs - sn * sn) + a * u * cs + b2 * v * sn;
                    double step = gp > 0 ? g / gp : copysign(dtm, g);
                    t -= fmax(-dtm, fmin(dtm, step));
                }
                double sn, cs;
                sincos(t, &sn, &cs);
                dcur = sqrt((a * cs - u) * (a * cs - u) + (b2 * sn - v) * (b2 * sn - v));
                hloc = 2.0 * kPi * sqrt(a * a * sn * sn + b2 * b2 * cs * cs) / n;
                if (dcur < dbest && dcur > 0) {
                    // direction from the target to the closest point, back in the lab frame
                    const double ex = (a * cs - u) / dcur, ey = (b2 * sn - v) / dcur;
                    dbest = dcur;
                    dirx = ct * ex - st * ey;
                    diry = st * ex + ct * ey;
                }
            }
            if (dcur < gap_lim) atomicMin(gap_min, (unsigned long long)__double_as_longlong(dcur));
            if (!(sqrt(d2) < zone)) continue;
            // For a density of full bandwidth the rho-fold rule errs by about
            // exp(-(rho - 1/2) 2 pi d / h_loc): rho - 1/2 >= 6.4 h_loc / d puts it
            // below e^-40; rho >= 2 everywhere in the zone (the smooth rule,
            // rho = 1, errs by exp(-pi d / h), not negligible inside 10 h_b).
            int rho = 2;
            while ((rho - 0.5) * dcur < 6.4 * hloc && rho < kMaxRho) rho <<= 1;
            if ((rho - 0.5) * dcur < 6.4 * hloc) atomicAdd(overflow + 1, 1);  // closer than kMaxRho resolves
            if (imc) {
                // image (m, n) of body b seen from the translate of the target
                const int m = (im % 3 - 1) + (wi % 3 - 1), nn = (im / 3 - 1) + (wi / 3 - 1);
                const int4 r = bimg[b];
                if (!(r.y <= m && m <= r.x + 1 && r.w <= nn && nn <= r.z + 1)) atomicOr(gflag, 2);
            }
            if (c < kmax) {
                slots[(size_t)i * kmax + c] = make_int4(b, im, rho, 0);
                atomicMax(rho_max, rho);
            }
            ++c;
        }
    }
    if (c > kmax) {
        atomicMax(overflow, c);
        c = kmax;
    }
    count[i] = c;
    dmin[i] = (float)dbest;
    ddir[i] = make_float2((float)dirx, (float)diry);
}

// Exclusive scan (one CTA) of the per-target pair counts and of the block
// sizes 3 N_b per pair: pair_base[i], and per pair its block offset.
__global__ void k_close_scan(const int* __restrict__ count, int N, int kmax, const int4* __restrict__ slots,
                             const double* __restrict__ body, int* __restrict__ pair_base,
                             long long* __restrict__ blk_off, int4* __restrict__ pairs, int* __restrict__ totals,
                             long long* __restrict__ total_doubles, long long cap_doubles, int cap_pairs) {
    __shared__ int s_cnt[1024];
    __shared__ long long s_sz[1024];
    int tid = threadIdx.x, nt = blockDim.x;
    int per = (N + nt - 1) / nt;
    int lo = min(N, tid * per), hi = min(N, lo + per);
    int c = 0;
    long long sz = 0;
    for (int i = lo; i < hi; ++i) {
        c += count[i];
        for (int k = 0; k < count[i]; ++k) sz += 3 * (long long)body[8 * slots[(size_t)i * kmax + k].x + 5];
    }
    s_cnt[tid] = c;
    s_sz[tid] = sz;
    __syncthreads();
    if (tid == 0) {
        int a = 0;
        long long b = 0;
        for (int t = 0; t < nt; ++t) {
            int ca = s_cnt[t];
            long long sb = s_sz[t];
            s_cnt[t] = a;
            s_sz[t] = b;
            a += ca;
            b += sb;
        }
        totals[0] = a;
        totals[1] = (b > cap_doubles || a > cap_pairs) ? 1 : 0;
        *total_doubles = b;
    }
    __syncthreads();
    int p = s_cnt[tid];
    long long o = s_sz[tid];
    for (int i = lo; i < hi; ++i) {
        pair_base[i] = p;
        for (int k = 0; k < count[i]; ++k) {
            int4 sl = slots[(size_t)i * kmax + k];
            if (p < cap_pairs && o + 3 * (long long)body[8 * sl.x + 5] <= cap_doubles) {
                pairs[p] = make_int4(i, sl.x, sl.y, sl.z);
                blk_off[p] = o;
            }
            ++p;
            o += 3 * (long long)body[8 * sl.x + 5];
        }
    }
    if (tid == nt - 1) pair_base[N] = p;
}

// Dirichlet kernel tables D(2 pi j / (rho n)), j < rho n, of the n-point
// interpolant, for rho = 2, 4, ..., rho_max: table (n, rho) starts at
// base + n (rho - 2).  One thread per entry.
__global__ void k_dirichlet(double* __restrict__ tab, int n, int rho_max) {
    long long total = (2LL * rho_max - 2) * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int rho = 2;
        long long base = 0;
        while (idx >= base + (long long)rho * n) {
            base += (long long)rho * n;
            rho <<= 1;
        }
        int f = (int)(idx - base), nf = rho * n;
        double dv;
        if (f == 0) dv = 1.0;
        else if (f % rho == 0) dv = 0.0;
        else dv = sinpi((double)f / rho) * cospi((double)f / nf) / (sinpi((double)f / nf) * n);
        tab[idx] = dv;
    }
}

constexpr int kCloseChunk = 2048;  // fine nodes staged in shared memory at a time

// One CTA per close pair and range of kCloseAccNodes source nodes
// (blockIdx.y).  The fine grid (rho N_b nodes) is streamed through shared
// memory in chunks; warp w accumulates C_k for k = k0 + w, k0 + w + 8, ...
// with its lanes on consecutive fine nodes (coalesced table and shared
// reads).  Dynamic shared memory: 3 kCloseChunk + 3 min(N_b, kCloseAccNodes)
// doubles.
__global__ void __launch_bounds__(256)
k_close_blocks(const int4* __restrict__ pairs, const long long* __restrict__ blk_off,
               const double* __restrict__ x, const double* __restrict__ y,
               const double* __restrict__ nx, const double* __restrict__ ny,
               const double* __restrict__ w, const double* __restrict__ body,
               const int* __restrict__ node_cell, const Cell* __restrict__ cells,
               const double* __restrict__ dtab, const long long* __restrict__ dtab_off,
               double* __restrict__ blocks, float* __restrict__ blocks32, const double* __restrict__ bshape) {
    extern __shared__ double sm[];
    double* sa = sm;
    double* sb = sm + kCloseChunk;
    double* sd = sm + 2 * kCloseChunk;
    double* acc = sm + 3 * kCloseChunk;
    int4 pr = pairs[blockIdx.x];
    int i = pr.x, b = pr.y, im = pr.z, rho = pr.w;
    const Cell& sh = cells[node_cell[i]];
    const double* bd = body + 8 * b;
    double a = bd[0], bb = bd[1], xc = bd[2] + sh.sx[im], yc = bd[3] + sh.sy[im], th = bd[4];
    int nbn = (int)bd[5], off = (int)bd[6];
    int nf = rho * nbn;
    const double* dir = dtab + dtab_off[b] + (long long)nbn * (rho - 2);
    double X = x[i], Y = y[i], n0 = nx[i], n1 = ny[i];
    double st, ct;
    sincos(th, &st, &ct);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k0 = blockIdx.y * kCloseAccNodes, nk = min(kCloseAccNodes, nbn - k0);
    if (nk <= 0) return;  // this body has fewer node ranges than the largest one
    for (int k = threadIdx.x; k < 3 * nk; k += blockDim.x) acc[k] = 0.0;
    for (int f0 = 0; f0 < nf; f0 += kCloseChunk) {
        int cnt = min(kCloseChunk, nf - f0);
        __syncthreads();
        const double* shp = bshape + 4 * b;
        for (int u = threadIdx.x; u < cnt; u += blockDim.x) {
            int f = f0 + u;
            double t = (2.0 * kPi * f) / nf;
            double s, c;
            sincos(t, &s, &c);
            double px = a * c, py = bb * s;
            double dpx = -a * s, dpy = bb * c;
            if (shp[0] == 1.0) {
                double ddpx, ddpy;
                star_curve(shp, t, px, py, dpx, dpy, ddpx, ddpy);
            }
            double yx = xc + (ct * px - st * py), yy = yc + (st * px + ct * py);
            double dx = ct * dpx - st * dpy, dy = st * dpx + ct * dpy;
            double wf = (2.0 * kPi / nf) * sqrt(dx * dx + dy * dy);
            double rx = X - yx, ry = Y - yy;
            double r2 = rx * rx + ry * ry;
            double cc = -(rx * n0 + ry * n1) * wf / (kPi * r2 * r2);
            sa[u] = cc * rx * rx;
            sb[u] = cc * rx * ry;
            sd[u] = cc * ry * ry;
        }
        __syncthreads();
        for (int kk = wid; kk < nk; kk += nw) {
            const int k = k0 + kk;
            double A = 0, B = 0, D = 0;
            int base = f0 - rho * k;
            for (int u = lane; u < cnt; u += 32) {
                int j = base + u;
                j += (j < 0) ? nf : 0;
                double dv = __ldg(dir + j);
                A = fma(sa[u], dv, A);
                B = fma(sb[u], dv, B);
                D = fma(sd[u], dv, D);
            }
            for (int o = 16; o > 0; o >>= 1) {
                A += __shfl_xor_sync(0xffffffffu, A, o);
                B += __shfl_xor_sync(0xffffffffu, B, o);
                D += __shfl_xor_sync(0xffffffffu, D, o);
            }
            if (lane == 0) {
                acc[3 * kk] += A;
                acc[3 * kk + 1] += B;
                acc[3 * kk + 2] += D;
            }
        }
    }
    __syncthreads();
    double* out = blocks + blk_off[blockIdx.x];
    for (int kk = threadIdx.x; kk < nk; kk += blockDim.x) {
        // minus the smooth rule's term for node k of this body image
        const int k = k0 + kk;
        double rx = X - (x[off + k] + sh.sx[im]), ry = Y - (y[off + k] + sh.sy[im]);
        double r2 = rx * rx + ry * ry;
        double cc = -(rx * n0 + ry * n1) * w[off + k] / (kPi * r2 * r2);
        const double A = acc[3 * kk] - cc * rx * rx;
        const double B = acc[3 * kk + 1] - cc * rx * ry;
        const double D = acc[3 * kk + 2] - cc * ry * ry;
        out[3 * k] = A;
        out[3 * k + 1] = B;
        out[3 * k + 2] = D;
        // single-precision copy acting on q = sigma w (the packed sources)
        const double iw = 1.0 / w[off + k];
        float* o32 = blocks32 + blk_off[blockIdx.x] + 3 * k;
        o32[0] = (float)(A * iw);
        o32[1] = (float)(B * iw);
        o32[2] = (float)(D * iw);
    }
}

// ---------------------------------------------------------------------------
// The paper's special quadrature (Sec. 6.3, opts.close_rule = 1).  In complex
// notation (z the target, n its normal, zeta the source point, s = sigma) the
// traction kernel of Eq. Gt is
//   -(1/4pi) [ conj(n) conj(s) r / conj(r)^2 + (conj(n) s + n conj(s)) / conj(r) + n s / r ],
// r = z - zeta, so the integral over a body's curve is made of the Cauchy
// integrals C[h](z) = (1/2 pi i) oint h / (zeta - z) dzeta (and C') of
// h = s / tau, conj(s) / tau, s conj(zeta) / tau.  For a target outside the
// curve C[h] is analytic outside it and vanishes at infinity: its boundary
// values phi = E h follow from the Plemelj formula with a smooth integrand,
//   E = (K + (2 pi / N) Dspec) / (2 pi i),  K_jk = wt_k / (zeta_k - zeta_j) (k != j),
//   K_jj = -sum_{k != j} K_jk,  wt_k = w_k tau_k = zeta'(t_k) 2 pi / N,
// Dspec the spectral differentiation matrix of the N-point interpolant
// (Dspec_jk = d[(j - k) mod N], d_m = (-1)^m cot(pi m / N) / 2 for even N,
// (-1)^m / (2 sin(pi m / N)) for odd N), and its value
// near the curve from the compensated exterior barycentric rule
//   C[h](z) = sum_j beta_j phi_j,  beta_j = W_j / (sum_i W_i - 2 pi i),  W_j = wt_j / (zeta_j - z);
// C'[h] the same with phi' = diag(1 / zeta') Dspec phi.  As a linear map of
// the nodal density this gives per node k, with a = E^T beta and
// b = E^T Dspec^T (beta / zeta'),
//   p_k = -2 pi i a_k conj(tau_k),  q_k = 2 pi i b_k (conj(z) - conj(zeta_k)) conj(tau_k),
//   alpha_k = -2 Re(n p_k) / (4 pi),  gamma_k = -(n conj(p_k) + conj(n) conj(q_k)) / (4 pi),
// T = sum_k alpha_k s_k + gamma_k conj(s_k): alpha is real, so the block of
// node k is the symmetric [[alpha + Re gamma, Im gamma], [Im gamma, alpha - Re gamma]]
// (the same storage as the fine rule's blocks), minus the smooth rule's term.
// All in FP64; O(N_b^2) per block whatever the target's distance.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// a / b
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double inv = 1.0 / (b.x * b.x + b.y * b.y);
    return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
// wt = w tau with the unit tangent tau = (-n_y, n_x) (the outward normal is tau turned clockwise)
__device__ __forceinline__ double2 node_wt(const double* w, const double* nx, const double* ny, int j) {
    return make_double2(-w[j] * ny[j], w[j] * nx[j]);
}

// Per body (one CTA each): K_kk = -sum_{m != k} wt_m / (zeta_m - zeta_k) (shift-
// invariant) and the body's spectral-derivative table d_m.
__global__ void __launch_bounds__(256)
k_bary_pre(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
           const double* __restrict__ ny, const double* __restrict__ w, const double* __restrict__ body,
           double2* __restrict__ kd, double* __restrict__ dcot) {
    const double* bd = body + 8 * blockIdx.x;
    const int n = (int)bd[5], off = (int)bd[6];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double zx = x[off + k], zy = y[off + k];
        double sr = 0.0, si = 0.0;
        for (int m = 0; m < n; ++m) {
            if (m == k) continue;
            const double2 q = cdiv(node_wt(w, nx, ny, off + m), make_double2(x[off + m] - zx, y[off + m] - zy));
            sr += q.x;
            si += q.y;
        }
        kd[off + k] = make_double2(-sr, -si);
        // even N (bie_init requires it): cot, the Nyquist mode's derivative zero at the
        // nodes; odd N would take csc
        const double sg = (k & 1) ? -1.0 : 1.0;
        dcot[off + k] = k == 0 ? 0.0 : 0.5 * sg / ((n & 1) ? sin(kPi * k / n) : tan(kPi * k / n));
    }
}

constexpr int kBaryTile = 256;

// One CTA per (target, body image) pair: the block of every node of the body
// image by the barycentric rule.  scratch holds a_k and u_k = (Dspec^T (beta /
// zeta'))_k per node (2 double2 at 2 (blk_off / 3 + k)).
__global__ void __launch_bounds__(kBaryTile)
k_close_blocks_bary(const int4* __restrict__ pairs, const long long* __restrict__ blk_off,
                    const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ nx,
                    const double* __restrict__ ny, const double* __restrict__ w, const double* __restrict__ body,
                    const int* __restrict__ node_cell, const Cell* __restrict__ cells,
                    const double2* __restrict__ kd, const double* __restrict__ dcot, double2* __restrict__ scratch,
                    double* __restrict__ blocks, float* __restrict__ blocks32) {
    __shared__ double2 s_z[kBaryTile], s_v[kBaryTile], s_u[kBaryTile];
    __shared__ double red[2][kBaryTile / 32];
    const int4 pr = pairs[blockIdx.x];
    const int i = pr.x, b = pr.y, im = pr.z;
    const Cell& cl = cells[node_cell[i]];
    const double* bd = body + 8 * b;
    const int n = (int)bd[5], off = (int)bd[6];
    const double sx = cl.sx[im], sy = cl.sy[im];
    const double2 z = make_double2(x[i], y[i]);
    const double2 nn = make_double2(nx[i], ny[i]);
    const long long bo = blk_off[blockIdx.x];
    double2* sc = scratch + 2 * (bo / 3);
    const int t = threadIdx.x;
    const double two_pi = 2.0 * kPi;
    // S' = sum_j W_j - 2 pi i (fixed-order block reduction)
    double sr = 0.0, si = 0.0;
    for (int j = t; j < n; j += kBaryTile) {
        const double2 q = cdiv(node_wt(w, nx, ny, off + j), make_double2(x[off + j] + sx - z.x, y[off + j] + sy - z.y));
        sr += q.x;
        si += q.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((t & 31) == 0) {
        red[0][t >> 5] = sr;
        red[1][t >> 5] = si;
    }
    __syncthreads();
    double2 Sp = make_double2(0.0, 0.0);
    for (int k = 0; k < kBaryTile / 32; ++k) {
        Sp.x += red[0][k];
        Sp.y += red[1][k];
    }
    Sp.y -= two_pi;
    auto beta = [&](int j, double2 zj) {  // W_j / S'
        return cdiv(cdiv(node_wt(w, nx, ny, off + j), make_double2(zj.x - z.x, zj.y - z.y)), Sp);
    };
    auto zeta = [&](int j) { return make_double2(x[off + j] + sx, y[off + j] + sy); };
    const double scale = two_pi / n;
    // pass 1: a = E^T beta and u = Dspec^T (beta / zeta'), zeta' = wt / scale
    for (int kc = 0; kc < n; kc += kBaryTile) {
        const int k = kc + t;
        const bool valid = k < n;
        const double2 zk = valid ? zeta(k) : make_double2(0.0, 0.0);
        double2 aA = make_double2(0, 0), aD = make_double2(0, 0), aU = make_double2(0, 0);
        for (int jt = 0; jt < n; jt += kBaryTile) {
            __syncthreads();
            const int j = jt + t;
            if (j < n) {
                const double2 zj = zeta(j);
                const double2 bj = beta(j, zj);
                s_z[t] = zj;
                s_v[t] = bj;
                s_u[t] = cdiv(cmul(bj, make_double2(scale, 0.0)), node_wt(w, nx, ny, off + j));  // beta / zeta'
            }
            __syncthreads();
            if (!valid) continue;
            const int cnt = min(kBaryTile, n - jt);
            for (int jj = 0; jj < cnt; ++jj) {
                const int jg = jt + jj;
                const double2 bj = s_v[jj];
                if (jg != k) {
                    const double2 r = cdiv(bj, make_double2(zk.x - s_z[jj].x, zk.y - s_z[jj].y));
                    aA.x += r.x;
                    aA.y += r.y;
                }
                int m = jg - k;
                m += m < 0 ? n : 0;
                const double dd = dcot[off + m];
                aD.x = fma(dd, bj.x, aD.x);
                aD.y = fma(dd, bj.y, aD.y);
                aU.x = fma(dd, s_u[jj].x, aU.x);
                aU.y = fma(dd, s_u[jj].y, aU.y);
            }
        }
        if (valid) {
            const double2 bk = beta(k, zk);
            double2 v = cmul(node_wt(w, nx, ny, off + k), aA);
            const double2 kb = cmul(kd[off + k], bk);
            v.x += kb.x + scale * aD.x;
            v.y += kb.y + scale * aD.y;
            sc[2 * k] = make_double2(v.y / two_pi, -v.x / two_pi);  // v / (2 pi i)
            sc[2 * k + 1] = aU;
        }
    }
    __syncthreads();
    // pass 2: b = E^T u, then the node blocks
    for (int kc = 0; kc < n; kc += kBaryTile) {
        const int k = kc + t;
        const bool valid = k < n;
        const double2 zk = valid ? zeta(k) : make_double2(0.0, 0.0);
        double2 aB = make_double2(0, 0), aE = make_double2(0, 0);
        for (int jt = 0; jt < n; jt += kBaryTile) {
            __syncthreads();
            const int j = jt + t;
            if (j < n) {
                s_z[t] = zeta(j);
                s_u[t] = sc[2 * j + 1];
            }
            __syncthreads();
            if (!valid) continue;
            const int cnt = min(kBaryTile, n - jt);
            for (int jj = 0; jj < cnt; ++jj) {
                const int jg = jt + jj;
                const double2 uj = s_u[jj];
                if (jg != k) {
                    const double2 r = cdiv(uj, make_double2(zk.x - s_z[jj].x, zk.y - s_z[jj].y));
                    aB.x += r.x;
                    aB.y += r.y;
                }
                int m = jg - k;
                m += m < 0 ? n : 0;
                const double dd = dcot[off + m];
                aE.x = fma(dd, uj.x, aE.x);
                aE.y = fma(dd, uj.y, aE.y);
            }
        }
        if (!valid) continue;
        const double2 wtk = node_wt(w, nx, ny, off + k);
        double2 v = cmul(wtk, aB);
        const double2 ku = cmul(kd[off + k], sc[2 * k + 1]);
        v.x += ku.x + scale * aE.x;
        v.y += ku.y + scale * aE.y;
        const double2 bk = make_double2(v.y / two_pi, -v.x / two_pi);
        const double2 ak = sc[2 * k];
        const double2 tauc = make_double2(-ny[off + k], -nx[off + k]);  // conj(tau)
        // p = -2 pi i a conj(tau), q = 2 pi i b (conj(z) - conj(zeta_k)) conj(tau)
        const double2 at = cmul(ak, tauc);
        const double2 p = make_double2(two_pi * at.y, -two_pi * at.x);
        const double2 bt = cmul(cmul(bk, make_double2(z.x - zk.x, -(z.y - zk.y))), tauc);
        const double2 q = make_double2(-two_pi * bt.y, two_pi * bt.x);
        const double al = -2.0 * (nn.x * p.x - nn.y * p.y) / (4.0 * kPi);
        const double2 g1 = cmul(nn, cconj(p)), g2 = cmul(cconj(nn), cconj(q));
        const double gr = -(g1.x + g2.x) / (4.0 * kPi), gi = -(g1.y + g2.y) / (4.0 * kPi);
        // minus the smooth rule's term for node k of this body image
        const double rx = z.x - zk.x, ry = z.y - zk.y;
        const double r2 = rx * rx + ry * ry;
        const double cc = -(rx * nn.x + ry * nn.y) * w[off + k] / (kPi * r2 * r2);
        const double A = al + gr - cc * rx * rx;
        const double B = gi - cc * rx * ry;
        const double D = al - gr - cc * ry * ry;
        double* out = blocks + bo + 3 * k;
        out[0] = A;
        out[1] = B;
        out[2] = D;
        const double iw = 1.0 / w[off + k];
        float* o32 = blocks32 + bo + 3 * k;
        o32[0] = (float)(A * iw);
        o32[1] = (float)(B * iw);
        o32[2] = (float)(D * iw);
    }
}

// One warp per target: T_i += sum over its pairs of C sigma_b (slot order).
__global__ void k_close_apply(const int* __restrict__ pair_base, const int4* __restrict__ pairs,
                              const long long* __restrict__ blk_off, const double* __restrict__ blocks,
                              const double* __restrict__ body, const double2* __restrict__ sigma, int N,
                              double2* __restrict__ T) {
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= N) return;
    int p0 = pair_base[wid], p1 = pair_base[wid + 1];
    if (p0 == p1) return;
    double tx = 0, ty = 0;
    for (int p = p0; p < p1; ++p) {
        int b = pairs[p].y;
        int nbn = (int)body[8 * b + 5], off = (int)body[8 * b + 6];
        const double* C = blocks + blk_off[p];
        double ax = 0, ay = 0;
        for (int k = lane; k < nbn; k += 32) {
            double2 s = sigma[off + k];
            double A = C[3 * k], B = C[3 * k + 1], D = C[3 * k + 2];
            ax = fma(A, s.x, fma(B, s.y, ax));
            ay = fma(B, s.x, fma(D, s.y, ay));
        }
        for (int o = 16; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        tx += ax;
        ty += ay;
    }
    if (lane == 0) {
        double2 t = T[wid];
        T[wid] = make_double2(t.x + tx, t.y + ty);
    }
}

// Replace *p by a fresh device array of count elements (the old contents are
// not kept).
template <typename T>
static int regrow(bie_ctx* c, T** p, size_t count) {
    if (*p) BIE_CUDA(c, cudaFree(*p));
    *p = nullptr;
    BIE_CUDA(c, cudaMalloc((void**)p, count * sizeof(T) + 16));
    return BIE_OK;
}

// The doubled-cell periodizer's geometry conditions (flags[7], set by
// k_geometry and k_close_detect).
static int doubled_cell_check(bie_ctx* c, int f) {
    if (f & 1)
        return fail(c, BIE_EINVAL, "n_images 4: a node lies beyond the doubled cell (a body larger than the cell?)");
    if (f & 2)
        return fail(c, BIE_EINVAL, "n_images 4: a close-evaluation pair sees a body image that is not among all its "
                                   "nodes' doubled-cell images (a body larger than about half a cell)");
    return BIE_OK;
}

int build_close(bie_ctx* c) {
    ++c->epoch;  // close pairs, blocks and their storage change
    c->cl.npairs = 0;
    c->cl.rho_max = 0;
    k_body_h<<<c->nb, 256, 0, c->stream>>>(c->w, c->body);
    BIE_LAUNCH(c, "k_body_h");
    c->cl.min_gap = INFINITY;
    const double gap_lim = c->opts.min_gap > 0 ? c->opts.min_gap : 0.0;
    if (!(c->opts.close_factor > 0) && !(gap_lim > 0)) {
        if (c->utilde) {
            int f = 0;
            BIE_CUDA(c, cudaMemcpyAsync(&f, c->cl.flags + 7, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            BIE_CUDA(c, cudaStreamSynchronize(c->stream));
            return doubled_cell_check(c, f);
        }
        return BIE_OK;
    }
    const int N = c->N, kmax = kCloseSlots;
    BIE_CUDA(c, cudaMemsetAsync(c->cl.flags, 0, 4 * sizeof(int), c->stream));
    BIE_CUDA(c, cudaMemsetAsync(c->cl.flags + 6, 0, sizeof(int), c->stream));
    unsigned long long* gap_min = reinterpret_cast<unsigned long long*>(c->cl.flags + 4);
    long long* need = reinterpret_cast<long long*>(c->cl.flags + 8);
    BIE_CUDA(c, cudaMemsetAsync(gap_min, 0xFF, sizeof(unsigned long long), c->stream));
    k_close_detect<<<(N + 127) / 128, 128, 0, c->stream>>>(c->x, c->y, c->owner, c->body, c->node_cell, c->cells, N,
                                                         c->opts.close_factor, gap_lim, kmax, c->cl.slots,
                                                         c->cl.count, c->cl.flags + 2, gap_min, c->cl.flags + 6,
                                                         c->cl.dmin, c->cl.ddir, c->utilde ? c->imc : nullptr,
                                                         c->bimg, c->cl.flags + 7, c->bshape);
    BIE_LAUNCH(c, "k_close_detect");
    int h[8];
    long long need_doubles = 0;
    unsigned long long gm = 0;
    // the scan again after growing the storage (never a third time: the
    // second pass is sized from the first's totals)
    for (int pass = 0; pass < 2; ++pass) {
        k_close_scan<<<1, 1024, 0, c->stream>>>(c->cl.count, N, kmax, c->cl.slots, c->body, c->cl.pair_base,
                                               c->cl.blk_off, c->cl.pairs, c->cl.flags, need, c->cl.cap_doubles,
                                               c->cl.cap_pairs);
        BIE_LAUNCH(c, "k_close_scan");
        BIE_CUDA(c, cudaMemcpyAsync(h, c->cl.flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        BIE_CUDA(c, cudaMemcpyAsync(&need_doubles, need, sizeof need_doubles, cudaMemcpyDeviceToHost, c->stream));
        BIE_CUDA(c, cudaMemcpyAsync(&gm, gap_min, sizeof gm, cudaMemcpyDeviceToHost, c->stream));
        BIE_CUDA(c, cudaStreamSynchronize(c->stream));
        if (int rc = doubled_cell_check(c, h[7])) return rc;
        if (h[2] > 0)
            return fail(c, BIE_EINVAL, "a node is close to more than " + std::to_string(kmax) +
                                           " body images (bodies overlap or nearly so)");
        if (!h[1]) break;
        if (!c->cl.grow || pass == 1)
            return fail(c, BIE_EINVAL, "close-evaluation storage exceeded (" + std::to_string(h[0]) +
                                           " pairs); raise close_capacity");
        // grow by a quarter beyond what this geometry needs
        if (h[0] > c->cl.cap_pairs) {
            const int cap = h[0] + h[0] / 4 + 16;
            int rc = regrow(c, &c->cl.pairs, cap);
            rc = rc ? rc : regrow(c, &c->cl.blk_off, cap);
            if (rc) return rc;
            c->cl.cap_pairs = cap;
        }
        if (need_doubles > c->cl.cap_doubles) {
            const long long cap = need_doubles + need_doubles / 4 + 1024;
            int rc = regrow(c, &c->cl.blocks, (size_t)cap);
            rc = rc ? rc : regrow(c, &c->cl.blocks32, (size_t)cap);
            if (!rc && c->cl.rule == 1) {
                rc = regrow(c, &c->cl.bary, (size_t)(2 * (cap / 3) + 2));
                c->cl.cap_bary = 2 * (cap / 3) + 2;
            }
            if (rc) return rc;
            c->cl.cap_doubles = cap;
        }
    }
    if (gm != ~0ULL) std::memcpy(&c->cl.min_gap, &gm, sizeof gm);
    c->cl.under_resolved = c->cl.rule == 1 ? 0 : h[3];  // the barycentric rule has no finest factor
    c->cl.npairs = h[0];
    c->cl.rho_max = h[6];
    if (h[0] == 0) return BIE_OK;
    if (c->cl.rule == 1) {
        k_bary_pre<<<c->nb, 256, 0, c->stream>>>(c->x, c->y, c->nx, c->ny, c->w, c->body, c->cl.bkd, c->cl.bcot);
        BIE_LAUNCH(c, "k_bary_pre");
        k_close_blocks_bary<<<h[0], kBaryTile, 0, c->stream>>>(c->cl.pairs, c->cl.blk_off, c->x, c->y, c->nx,
                                                              c->ny, c->w, c->body, c->node_cell, c->cells,
                                                              c->cl.bkd, c->cl.bcot, c->cl.bary, c->cl.blocks,
                                                              c->cl.blocks32);
        BIE_LAUNCH(c, "k_close_blocks_bary");
        return BIE_OK;
    }
    if (h[6] > c->cl.dtab_rho) {
        int rc = build_dirichlet_tables(c, h[6]);
        if (rc) return rc;
    }
    int maxn = 0;
    for (int n : c->n_nodes) maxn = std::max(maxn, n);
    const int acc = std::min(maxn, kCloseAccNodes);
    size_t shm = sizeof(double) * (3 * (size_t)kCloseChunk + 3 * (size_t)acc);
    BIE_CUDA(c, cudaFuncSetAttribute(k_close_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    c->cl.shm_limit = shm;
    dim3 grid(h[0], (maxn + kCloseAccNodes - 1) / kCloseAccNodes);
    k_close_blocks<<<grid, 256, shm, c->stream>>>(c->cl.pairs, c->cl.blk_off, c->x, c->y, c->nx, c->ny, c->w,
                                                  c->body, c->node_cell, c->cells, c->cl.dtab, c->cl.dtab_off,
                                                  c->cl.blocks, c->cl.blocks32, c->bshape);
    BIE_LAUNCH(c, "k_close_blocks");
    return BIE_OK;
}

// Dirichlet tables for every distinct node count, rho = 2 .. rho_max
// (rebuilt, larger, when a geometry needs a finer rule than they hold).
int build_dirichlet_tables(bie_ctx* c, int rho_max) {
    rho_max = std::max(rho_max, 64);
    std::vector<long long> off(c->nb);
    std::vector<std::pair<int, long long>> seen;
    long long total = 0;
    for (int b = 0; b < c->nb; ++b) {
        int n = c->n_nodes[b];
        long long o = -1;
        for (auto& pr : seen)
            if (pr.first == n) o = pr.second;
        if (o < 0) {
            o = total;
            seen.push_back({n, o});
            total += (2LL * rho_max - 2) * n;
        }
        off[b] = o;
    }
    int rc = regrow(c, &c->cl.dtab, (size_t)total);
    if (rc) return rc;
    if (!c->cl.dtab_off) BIE_CUDA(c, cudaMalloc((void**)&c->cl.dtab_off, c->nb * sizeof(long long)));
    BIE_CUDA(c, cudaMemcpyAsync(c->cl.dtab_off, off.data(), c->nb * sizeof(long long), cudaMemcpyHostToDevice,
                                c->stream));
    for (auto& pr : seen) {
        k_dirichlet<<<1024, 256, 0, c->stream>>>(c->cl.dtab + pr.second, pr.first, rho_max);
        BIE_LAUNCH(c, "k_dirichlet");
    }
    // the host vector `off` must outlive the asynchronous copy
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    c->cl.dtab_rho = rho_max;
    return BIE_OK;
}

// Single-precision assembly (a5 + a6 + a7 of one application), one warp
// per target: the traction T_i is summed from
//   - the target's near-sum partials (one per source split, TwoSum per lane),
//   - the proxy traction sum_p G^t(x_i, y_p; n_i) xi_p (single precision),
//   - the on-curve diagonal -(kappa_i / 2 pi) tau_i (tau_i . q_i),
//   - the close-evaluation corrections below,
// and the output is y_i = sigma_i / 2 + T_i + alpha n_i + F_b + (x_i - x^c)^perp tau_b
// with alpha = -T(x_1) . n_1 per cell (Sec. 6.2 remark on the pressure).
//
// Close-evaluation corrections.  k_near32 sums every pair from single-
// precision positions relative to the cell centre, whose rounding (~1e-7 of
// the cell size) is a large relative error in r = x_i - y_j for nodes close
// to the target, and larger still in r . n_i for the nearly tangent r between
// neighbours on one curve.  For the target's own body (unshifted) and for
// each of its close (body, image) pairs, the single-precision terms are
// recomputed bit for bit (same inputs, same pair32) and replaced by the same
// terms with r formed exactly from double-float positions (then rounded to
// single precision); the close-evaluation blocks are applied in single
// precision (stored divided by the weights, acting on q = sigma w).
// Everything but the final sums runs on the FP32 pipe.
//
// With the doubled-cell periodizer (imc non-null) the near sum evaluated the
// pair at the target's translate inside U (tgt32) against the source's image
// record src32[4 j + k], k the node's image that lands the body image where
// it is seen from that translate; the redo recomputes that term.
struct Asm32 {
    const float2* part;
    const float2* ypf;
    const float* xif;
    int M;
    const int* pair_base;
    const int4* pairs;
    const long long* blk_off;
    const float* blocks32;
    int use_pairs;
    const double* body;
    const int* owner;
    const double2* sigma;
    int N;
    const float4* tgt32;
    const float4* src32;
    const float4* posdf;
    const double* x;
    const double* y;
    const double* nx;
    const double* ny;
    const double* w;
    const double* kap;
    const int* node_cell;
    const Cell* cells;
    const int* imc;
    const double* bodyF;
};

// T_i on every thread of the calling group of NL threads (a warp, NL = 32,
// or a whole CTA, NL = blockDim.x = 256; red: 6 NL / 32 doubles of shared
// memory for NL > 32); fixed reduction order.
template <int NL>
__device__ __forceinline__ double2 traction32(const Asm32& a, int i, int lane, double* red) {
    const int cidx = a.node_cell[i];
    const Cell& cl = a.cells[cidx];
    // near-sum partials
    float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f, e;
    const int splits = cl.splits[0];
    const long long base = cl.part_off[0] + (i - cl.node_off);
    for (int s = lane; s < splits; s += NL) {
        const float2 p = a.part[base + (long long)s * cl.n_nodes];
        two_sum(hx, p.x, hx, e);
        lx += e;
        two_sum(hy, p.y, hy, e);
        ly += e;
    }
    // proxy traction
    const float4 tv = a.tgt32[i];
    const float2* yp = a.ypf + (size_t)cidx * a.M;
    const float* xi = a.xif + (size_t)cidx * 2 * a.M;
    float cx = 0.f, cy = 0.f;
    for (int p = lane; p < a.M; p += NL) {
        const float2 q = yp[p];
        const float rx = tv.x - q.x, ry = tv.y - q.y;
        const float fx = xi[p], fy = xi[a.M + p];
        const float inv = rcp_approx(fmaf(rx, rx, ry * ry));
        const float cc = (fmaf(rx, tv.z, ry * tv.w) * inv) * (fmaf(rx, fx, ry * fy) * inv);
        cx = fmaf(cc, rx, cx);
        cy = fmaf(cc, ry, cy);
    }
    // close-evaluation corrections
    const float4 pi = a.posdf[i];
    const int wi = a.imc ? img_wrap(a.imc[i]) : 4;
    float fx = 0.f, fy = 0.f;  // sum of (exactly differenced term - single-precision term)
    // target minus the image shift, exactly, as a double-float pair (xh, xl, yh, yl)
    auto shifted = [&](int im) {
        float4 p;
        df_diff(pi.x, pi.y, cl.sxf[im], cl.sxl[im], p.x, p.y);
        df_diff(pi.z, pi.w, cl.syf[im], cl.syl[im], p.z, p.w);
        return p;
    };
    auto redo = [&](int j, int im, const float4& p) {
        float4 s;
        float dx, dy;
        if (a.imc) {
            // image (m, n) of node j seen from the translate: its record index
            const int code = a.imc[j];
            const int dm = (im % 3 - 1) + (wi % 3 - 1) - img_m0(code);
            const int dn = (im / 3 - 1) + (wi / 3 - 1) - img_n0(code);
            // not among the node's images: the near sum has no such term (on
            // a body wider than half a cell, far from the target)
            if (dm < 0 || dm > 1 || dn < 0 || dn > 1) return;
            s = a.src32[4 * (size_t)j + (dm + 2 * dn)];
            dx = tv.x - s.x;
            dy = tv.y - s.y;
        } else {
            s = a.src32[j];
            dx = (tv.x - cl.sxf[im]) - s.x;
            dy = (tv.y - cl.syf[im]) - s.y;
        }
        const float c0 = pair32(dx, dy, tv.z, tv.w, s.z, s.w);
        const float4 q = a.posdf[j];
        float rh, rl, sh, sl;
        df_diff(p.x, p.y, q.x, q.y, rh, rl);
        df_diff(p.z, p.w, q.z, q.w, sh, sl);
        const float rx = rh + rl, ry = sh + sl;
        const float c1 = pair32(rx, ry, tv.z, tv.w, s.z, s.w);
        fx += c1 * rx - c0 * dx;
        fy += c1 * ry - c0 * dy;
    };
    {
        const int b = a.owner[i];
        const int nbn = (int)a.body[8 * b + 5], off = (int)a.body[8 * b + 6];
        const float4 p = shifted(4);
#pragma unroll 4
        for (int k = lane; k < nbn; k += NL)
            if (off + k != i) redo(off + k, 4, p);
    }
    float bx = 0.f, by = 0.f;  // close-evaluation blocks applied to q
    if (a.use_pairs) {
        const int p0 = a.pair_base[i], p1 = a.pair_base[i + 1];
        for (int pp = p0; pp < p1; ++pp) {
            const int4 pr = a.pairs[pp];
            const int b = pr.y, im = pr.z;
            const int nbn = (int)a.body[8 * b + 5], off = (int)a.body[8 * b + 6];
            const float* C = a.blocks32 + a.blk_off[pp];
            const float4 p = shifted(im);
#pragma unroll 2
            for (int k = lane; k < nbn; k += NL) {
                redo(off + k, im, p);
                const float4 s = a.src32[a.imc ? 4 * (size_t)(off + k) : (size_t)(off + k)];  // q: the same in every record
                const float A = C[3 * k], B = C[3 * k + 1], D = C[3 * k + 2];
                bx = fmaf(A, s.z, fmaf(B, s.w, bx));
                by = fmaf(B, s.z, fmaf(D, s.w, by));
            }
        }
    }
    const double c = -1.0 / kPi;
    double tx = (double)hx + (double)lx + c * (double)cx;
    double ty = (double)hy + (double)ly + c * (double)cy;
    for (int o = 16; o > 0; o >>= 1) {
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        ty += __shfl_xor_sync(0xffffffffu, ty, o);
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
    }
    if constexpr (NL > 32) {  // the warps' sums, added in warp order
        constexpr int nw = NL / 32;
        const int wid = lane >> 5;
        if ((lane & 31) == 0) {
            red[wid] = tx;
            red[nw + wid] = ty;
            red[2 * nw + wid] = fx;
            red[3 * nw + wid] = fy;
            red[4 * nw + wid] = bx;
            red[5 * nw + wid] = by;
        }
        __syncthreads();
        tx = ty = 0.0;
        double sfx = 0.0, sfy = 0.0, sbx = 0.0, sby = 0.0;
        for (int k = 0; k < nw; ++k) {
            tx += red[k];
            ty += red[nw + k];
            sfx += red[2 * nw + k];
            sfy += red[3 * nw + k];
            sbx += red[4 * nw + k];
            sby += red[5 * nw + k];
        }
        fx = (float)sfx;
        fy = (float)sfy;
        bx = (float)sbx;
        by = (float)sby;
    }
    // on-curve diagonal
    const double n0 = a.nx[i], n1 = a.ny[i];
    const double2 sg = a.sigma[i];
    const double t0 = -n1, t1 = n0;  // unit tangent
    const double qx = sg.x * a.w[i], qy = sg.y * a.w[i];
    const double dg = -(a.kap[i] / (2.0 * kPi)) * (t0 * qx + t1 * qy);
    return make_double2((tx + dg * t0) + (double)bx + c * (double)fx, (ty + dg * t1) + (double)by + c * (double)fy);
}

// alpha = -T(x_1) . n_1 of every cell (x_1: node 0 of its first body), one CTA per cell.
constexpr int kAlphaThreads = 256;
__global__ void __launch_bounds__(kAlphaThreads, 1) k_alpha32(Asm32 a, double* __restrict__ alpha) {
    __shared__ double red[6 * kAlphaThreads / 32];
    const int ci = blockIdx.x;
    const int i0 = a.cells[ci].node_off;
    const double2 T = traction32<kAlphaThreads>(a, i0, threadIdx.x, red);
    if (threadIdx.x == 0) alpha[ci] = -(T.x * a.nx[i0] + T.y * a.ny[i0]);
}

// y_i = sigma_i / 2 + T_i + alpha n_i + F_b + (x_i - x^c)^perp tau_b, one warp per target.
__global__ void __launch_bounds__(256, 3) k_assemble32(Asm32 a, const double* __restrict__ alpha,
                                                    double2* __restrict__ out) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= a.N) return;
    const double2 T = traction32<32>(a, i, lane, nullptr);
    if (lane != 0) return;
    const double al = alpha[a.node_cell[i]];
    const int b = a.owner[i];
    const double xc = a.body[8 * b + 2], yc = a.body[8 * b + 3];
    const double Fx = a.bodyF[3 * b], Fy = a.bodyF[3 * b + 1], tq = a.bodyF[3 * b + 2];
    const double2 s = a.sigma[i];
    const double ox = 0.5 * s.x + T.x + al * a.nx[i] + Fx - (a.y[i] - yc) * tq;
    const double oy = 0.5 * s.y + T.y + al * a.ny[i] + Fy + (a.x[i] - xc) * tq;
    out[i] = make_double2(ox, oy);
}

int assemble32(bie_ctx* c, const double* sigma, const Workspace& ws, double* yout) {
    Asm32 a;
    a.part = (const float2*)ws.part;
    a.ypf = c->ypf;
    a.xif = ws.xif;
    a.M = c->M;
    a.pair_base = c->cl.pair_base;
    a.pairs = c->cl.pairs;
    a.blk_off = c->cl.blk_off;
    a.blocks32 = c->cl.blocks32;
    a.use_pairs = c->cl.npairs > 0 ? 1 : 0;
    a.body = c->body;
    a.owner = c->owner;
    a.sigma = reinterpret_cast<const double2*>(sigma);
    a.N = c->N;
    a.tgt32 = c->tgt32;
    a.src32 = ws.src32;
    a.posdf = c->posdf;
    a.x = c->x;
    a.y = c->y;
    a.nx = c->nx;
    a.ny = c->ny;
    a.w = c->w;
    a.kap = c->kap;
    a.node_cell = c->node_cell;
    a.cells = c->cells;
    a.imc = c->utilde ? c->imc : nullptr;
    a.bodyF = ws.bodyF;
    double* alpha = ws.T;  // the single-precision path keeps no T: its first ncell entries hold alpha
    k_alpha32<<<c->ncell, kAlphaThreads, 0, c->stream>>>(a, alpha);
    BIE_LAUNCH(c, "k_alpha32");
    const int bs = 256;
    const int gs = (int)((32LL * c->N + bs - 1) / bs);
    k_assemble32<<<gs, bs, 0, c->stream>>>(a, alpha, reinterpret_cast<double2*>(yout));
    BIE_LAUNCH(c, "k_assemble32");
    return BIE_OK;
}

int close_apply(bie_ctx* c, const double* sigma, double* T) {
    if (c->cl.npairs == 0) return BIE_OK;
    const int bs = 256;
    const int gs = (int)((32LL * c->N + bs - 1) / bs);
    k_close_apply<<<gs, bs, 0, c->stream>>>(c->cl.pair_base, c->cl.pairs, c->cl.blk_off, c->cl.blocks, c->body,
                                           reinterpret_cast<const double2*>(sigma), c->N,
                                           reinterpret_cast<double2*>(T));
    BIE_LAUNCH(c, "k_close_apply");
    return BIE_OK;
}

}  // namespace bie
