// Per-geometry precompute: boundary nodes (Sec. 6, trapezoidal rule on each
// ellipse) and, per cell, the proxy-Stokeslet least-squares operator of
// Sec. 6.1.
//
// The proxy fit solves min |Q xi - d|^2 + lam^2 |xi|^2 (lam = lam_rel ||Q||_F),
// i.e. the least-squares problem of the stacked matrix [Q; lam I], by
// Householder QR in double precision.  The explicit operator P with
// xi = P d is formed once per geometry so that each operator application
// needs a single small matrix-vector product.  Cells are independent: every
// kernel runs over all cells of the batch at once (grid dimension "cell").
#include <cmath>

#include "bie_internal.cuh"

namespace bie {

// ---------------------------------------------------------------------------
// nodes, normals, weights, curvature
// ---------------------------------------------------------------------------
// With utilde (n_images 4) also each node's image code (Def. Gnear: the two
// integers m with -1 <= s + m < 1 are m0 = ceil(-1 - s) and m0 + 1, likewise
// n0 for t; (s, t) its lattice coordinates about the cell centre) and its
// translate into U (lattice coordinates rounded into [-1/2, 1/2)), where the
// periodic sums are evaluated (Sec. 6.2): xw, yw and tgt32 hold that
// translate.  A node whose images would leave the 3 x 3 shift table (a body
// reaching beyond the doubled cell) raises bit 0 of *gflag.
__global__ void k_geometry(const double* __restrict__ body, const int* __restrict__ owner,
                           const int* __restrict__ node_cell, const Cell* __restrict__ cells, int N,
                           double* __restrict__ x, double* __restrict__ y, double* __restrict__ nx,
                           double* __restrict__ ny, double* __restrict__ w, double* __restrict__ kap,
                           float4* __restrict__ tgt32, float4* __restrict__ posdf, int utilde,
                           double* __restrict__ xw, double* __restrict__ yw, int* __restrict__ imc,
                           int* __restrict__ gflag, const double* __restrict__ bshape) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* bd = body + 8 * owner[i];
    const Cell& cl = cells[node_cell[i]];
    double a = bd[0], b = bd[1], xc = bd[2], yc = bd[3], th = bd[4];
    int n = (int)bd[5], off = (int)bd[6];
    int k = i - off;
    double t = (2.0 * kPi * k) / n;
    double st, ct, s, c;
    sincos(t, &st, &ct);
    sincos(th, &s, &c);
    double px = a * ct, py = b * st, dpx = -a * st, dpy = b * ct, ddpx = -px, ddpy = -py;
    const double* shp = bshape + 4 * owner[i];
    if (shp[0] == 1.0) star_curve(shp, t, px, py, dpx, dpy, ddpx, ddpy);
    double X = xc + (c * px - s * py), Y = yc + (s * px + c * py);
    double dX = c * dpx - s * dpy, dY = s * dpx + c * dpy;
    double ddX = c * ddpx - s * ddpy, ddY = s * ddpx + c * ddpy;
    double sp = sqrt(dX * dX + dY * dY);
    double tx = dX / sp, ty = dY / sp;
    x[i] = X;
    y[i] = Y;
    nx[i] = ty;
    ny[i] = -tx;
    w[i] = (2.0 * kPi / n) * sp;
    kap[i] = (dX * ddY - dY * ddX) / (sp * sp * sp);
    double XW = X, YW = Y;
    if (utilde) {
        const double px_ = X - cl.C[0], py_ = Y - cl.C[1];
        const double ls = cl.inv[0] * px_ + cl.inv[1] * py_, lt = cl.inv[2] * px_ + cl.inv[3] * py_;
        const int m0 = (int)ceil(-1.0 - ls), n0 = (int)ceil(-1.0 - lt);
        const int wm = -(int)floor(ls + 0.5), wn = -(int)floor(lt + 0.5);
        if (m0 < -1 || m0 > 0 || n0 < -1 || n0 > 0 || wm < -1 || wm > 1 || wn < -1 || wn > 1) {
            atomicOr(gflag, 1);
            imc[i] = 0 | (0 << 1) | (4 << 2);
        } else {
            const int wi = (wn + 1) * 3 + (wm + 1);
            imc[i] = (m0 + 1) | ((n0 + 1) << 1) | (wi << 2);
            XW = X + cl.sx[wi];
            YW = Y + cl.sy[wi];
        }
    }
    xw[i] = XW;
    yw[i] = YW;
    tgt32[i] = make_float4((float)(XW - cl.C[0]), (float)(YW - cl.C[1]), (float)ty, (float)(-tx));
    float4 pd;
    split_df(X - cl.C[0], pd.x, pd.y);
    split_df(Y - cl.C[1], pd.z, pd.w);
    posdf[i] = pd;
}

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on (-1/2, 1/2) by Newton's method on P_m (host, once)
// ---------------------------------------------------------------------------
void gauss_legendre_half(int m, std::vector<double>& s) {
    s.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (m + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (m == 1) { p1 = z; p0 = 1.0; }
            double dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        s[m - 1 - i] = 0.5 * z;  // ascending order
    }
}

// ---------------------------------------------------------------------------
// proxy matrix Q (Sec. 6.1): rows [g1; g2; g3; g4] x (1-comps, 2-comps),
// columns (xi_1 of all proxies, xi_2 of all proxies); grid.y = cell
// ---------------------------------------------------------------------------
__device__ inline void stokeslet_d(double rx, double ry, double fx, double fy, double c4,
                                   double& ux, double& uy) {
    double r2 = rx * rx + ry * ry;
    double rf = (rx * fx + ry * fy) / r2;
    double l = -0.5 * log(r2);
    ux = (l * fx + rx * rf) * c4;
    uy = (l * fy + ry * rf) * c4;
}

__device__ inline void traction_d(double rx, double ry, double nx, double ny, double fx, double fy,
                                  double& tx, double& ty) {
    double r2 = rx * rx + ry * ry;
    double cc = -(rx * nx + ry * ny) * (rx * fx + ry * fy) / (kPi * r2 * r2);
    tx = cc * rx;
    ty = cc * ry;
}

__global__ void k_build_Q(double* __restrict__ A, int R, int m, int M, const double* __restrict__ gl_s,
                          const double* __restrict__ yp, const Cell* __restrict__ cells,
                          const double* __restrict__ e2v) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x, cidx = blockIdx.y;
    if (idx >= m * M) return;
    const Cell& cl = cells[cidx];
    const int l = idx % m, p = idx / m;
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = e2v[2 * cidx], e2y = e2v[2 * cidx + 1];
    const double Cx = cl.C[0], Cy = cl.C[1];
    double e1[2] = {e1x, e1y}, e2[2] = {e2x, e2y}, nl[2], nd[2];
    wall_normals(e1, e2, nl, nd);
    double s = gl_s[l];
    double xL = Cx - 0.5 * e1x + s * e2x, yL = Cy - 0.5 * e1y + s * e2y;
    double xD = Cx - 0.5 * e2x + s * e1x, yD = Cy - 0.5 * e2y + s * e1y;
    const double* ypc = yp + (size_t)cidx * 2 * M;
    double px = ypc[2 * p], py = ypc[2 * p + 1];
    double c4 = 1.0 / (4.0 * kPi * cl.mu);
    double* Ac = A + (size_t)cidx * R * 2 * M;
    for (int comp = 0; comp < 2; ++comp) {
        double fx = comp == 0 ? 1.0 : 0.0, fy = comp == 0 ? 0.0 : 1.0;
        double* col = Ac + (size_t)(comp * M + p) * R;
        double ua, va, ub, vb;
        // g1: velocity R - L
        stokeslet_d(xL + e1x - px, yL + e1y - py, fx, fy, c4, ua, va);
        stokeslet_d(xL - px, yL - py, fx, fy, c4, ub, vb);
        col[l] = ua - ub;
        col[m + l] = va - vb;
        // g2: traction R - L, normal nu_L
        traction_d(xL + e1x - px, yL + e1y - py, nl[0], nl[1], fx, fy, ua, va);
        traction_d(xL - px, yL - py, nl[0], nl[1], fx, fy, ub, vb);
        col[2 * m + l] = ua - ub;
        col[3 * m + l] = va - vb;
        // g3: velocity U - D
        stokeslet_d(xD + e2x - px, yD + e2y - py, fx, fy, c4, ua, va);
        stokeslet_d(xD - px, yD - py, fx, fy, c4, ub, vb);
        col[4 * m + l] = ua - ub;
        col[5 * m + l] = va - vb;
        // g4: traction U - D, normal nu_D
        traction_d(xD + e2x - px, yD + e2y - py, nd[0], nd[1], fx, fy, ua, va);
        traction_d(xD - px, yD - py, nd[0], nd[1], fx, fy, ub, vb);
        col[6 * m + l] = ua - ub;
        col[7 * m + l] = va - vb;
    }
}

__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread receives the result.  red: >= 33 doubles.
__device__ inline double block_sum(double v, double* red) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = lane < nw ? red[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// Householder QR of the stacked R x C matrix A = [Q; lam I] (column-major) of
// cell blockIdx.x, in place: the reflector v_k is stored in A[k:, k]
// (v_k[k] = A[k, k]), beta[k] its scalar, beta[C + k] the diagonal of the
// triangular factor.  One CTA per cell; the first Qrows rows hold Q on entry,
// the rest are filled here.
__global__ void k_qr(double* __restrict__ Aall, int R, int C, int Qrows, double lam_rel,
                     double* __restrict__ betaall) {
    __shared__ double red[33];
    double* A = Aall + (size_t)blockIdx.x * R * C;
    double* beta = betaall + (size_t)blockIdx.x * 2 * C;
    double* rdiag = beta + C;
    int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    double ss = 0.0;
    for (long long idx = tid; idx < (long long)Qrows * C; idx += nt) {
        int i = (int)(idx % Qrows), j = (int)(idx / Qrows);
        double a = A[i + (size_t)j * R];
        ss += a * a;
    }
    double lam = lam_rel * sqrt(block_sum(ss, red));
    int L = R - Qrows;
    for (long long idx = tid; idx < (long long)L * C; idx += nt) {
        int i = (int)(idx % L), j = (int)(idx / L);
        A[Qrows + i + (size_t)j * R] = (i == j) ? lam : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < C; ++k) {
        double* a = A + (size_t)k * R;
        double s = 0.0;
        for (int i = k + tid; i < R; i += nt) s += a[i] * a[i];
        s = block_sum(s, red);
        double akk = a[k];
        double nrm = sqrt(s);
        double alpha = akk > 0.0 ? -nrm : nrm;
        double v0 = akk - alpha;
        double vn2 = s - akk * akk + v0 * v0;
        double bk = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
        __syncthreads();
        if (tid == 0) {
            a[k] = v0;
            beta[k] = bk;
            rdiag[k] = alpha;
        }
        __syncthreads();
        for (int j = k + 1 + warp; j < C; j += nw) {
            double* aj = A + (size_t)j * R;
            double d = 0.0;
            for (int i = k + lane; i < R; i += 32) d += a[i] * aj[i];
            d = warp_sum(d) * bk;
            for (int i = k + lane; i < R; i += 32) aj[i] -= d * a[i];
        }
        __syncthreads();
    }
}

// Column c of P = first C rows of R^{-1} H_{C-1} ... H_0 e_c, c < Qrows, for
// cell blockIdx.y.  P is C x Qrows per cell, stored row-major
// (P[r * Qrows + c]) so that a warp reading one row of P in the operator
// application is coalesced.  Dynamic shared memory: R doubles.
__global__ void k_form_P(const double* __restrict__ Aall, int R, int C, const double* __restrict__ betaall,
                         double* __restrict__ Pall) {
    extern __shared__ double z[];
    __shared__ double red[33];
    const int Qrows = gridDim.x;
    const double* A = Aall + (size_t)blockIdx.y * R * C;
    const double* beta = betaall + (size_t)blockIdx.y * 2 * C;
    const double* rdiag = beta + C;
    double* P = Pall + (size_t)blockIdx.y * C * Qrows;
    int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < R; i += nt) z[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < C; ++k) {
        const double* a = A + (size_t)k * R;
        double d = 0.0;
        for (int i = k + tid; i < R; i += nt) d += a[i] * z[i];
        d = block_sum(d, red) * beta[k];
        for (int i = k + tid; i < R; i += nt) z[i] -= d * a[i];
        __syncthreads();
    }
    if (warp == 0) {
        for (int r = C - 1; r >= 0; --r) {
            double s = 0.0;
            for (int j = r + 1 + lane; j < C; j += 32) s += A[r + (size_t)j * R] * z[j];
            s = warp_sum(s);
            if (lane == 0) z[r] = (z[r] - s) / rdiag[r];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int r = tid; r < C; r += nt) P[(size_t)r * Qrows + c] = z[r];
}

// Per body the range of its nodes' image codes: (min m0, max m0, min n0,
// max n0); a body image (m, n) is wholly among its nodes' images when
// max m0 <= m <= min m0 + 1 and max n0 <= n <= min n0 + 1.
__global__ void k_body_img(const int* __restrict__ imc, const double* __restrict__ body, int4* __restrict__ bimg) {
    __shared__ int r[4];
    const int b = blockIdx.x;
    const int n = (int)body[8 * b + 5], off = (int)body[8 * b + 6];
    if (threadIdx.x == 0) {
        r[0] = 1;
        r[1] = -2;
        r[2] = 1;
        r[3] = -2;
    }
    __syncthreads();
    int a0 = 1, a1 = -2, b0 = 1, b1 = -2;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int code = imc[off + k];
        a0 = min(a0, img_m0(code));
        a1 = max(a1, img_m0(code));
        b0 = min(b0, img_n0(code));
        b1 = max(b1, img_n0(code));
    }
    atomicMin(&r[0], a0);
    atomicMax(&r[1], a1);
    atomicMin(&r[2], b0);
    atomicMax(&r[3], b1);
    __syncthreads();
    if (threadIdx.x == 0) bimg[b] = make_int4(r[0], r[1], r[2], r[3]);
}

int build_geometry(bie_ctx* c) {
    ++c->epoch;  // node data and the adopted proxy fit (pointers swapped by a time step)
    c->ws_x = nullptr;  // positions change: the workspace's sources are stale
    int bs = 256, gs = (c->N + bs - 1) / bs;
    int* gflag = c->cl.flags + 6 + 1;  // doubled-cell violations (read with the close pairs)
    BIE_CUDA(c, cudaMemsetAsync(gflag, 0, sizeof(int), c->stream));
    k_geometry<<<gs, bs, 0, c->stream>>>(c->body, c->owner, c->node_cell, c->cells, c->N, c->x, c->y, c->nx, c->ny,
                                        c->w, c->kap, c->tgt32, c->posdf, c->utilde ? 1 : 0, c->xw, c->yw, c->imc,
                                        gflag, c->bshape);
    BIE_LAUNCH(c, "k_geometry");
    if (c->utilde) {
        k_body_img<<<c->nb, 128, 0, c->stream>>>(c->imc, c->body, c->bimg);
        BIE_LAUNCH(c, "k_body_img");
    }
    return BIE_OK;
}

// Proxies on the walls of the doubled cell U~ (Sec. 6.1, remark after Eq. W):
// M / 4 per wall at the midpoints of equal sub-intervals, walls at lattice
// coordinates -1 and +1 about the cell centre (for side -1, then +1: the
// points C + side e1 + s e2, then C + side e2 + s e1).  grid.y = cell.
__global__ void k_proxy_box(int M, const Cell* __restrict__ cells, const double* __restrict__ e2v,
                            double* __restrict__ yp, float2* __restrict__ ypf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x, cidx = blockIdx.y;
    if (p >= M) return;
    const Cell& cl = cells[cidx];
    const int k = M / 4;
    const int side = p < 2 * k ? -1 : 1, q = p % (2 * k), j = q % k;
    const double s = (j + 0.5) / k * 2.0 - 1.0;
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = e2v[2 * cidx], e2y = e2v[2 * cidx + 1];
    double X, Y;
    if (q < k) {
        X = cl.C[0] + side * e1x + s * e2x;
        Y = cl.C[1] + side * e1y + s * e2y;
    } else {
        X = cl.C[0] + side * e2x + s * e1x;
        Y = cl.C[1] + side * e2y + s * e1y;
    }
    yp[(size_t)cidx * 2 * M + 2 * p] = X;
    yp[(size_t)cidx * 2 * M + 2 * p + 1] = Y;
    ypf[(size_t)cidx * M + p] = make_float2((float)(X - cl.C[0]), (float)(Y - cl.C[1]));
}

int build_proxy_fit_to(bie_ctx* c, ProxyFit& f, cudaStream_t st) {
    const int m = c->m, M = c->M;
    const int Qrows = 8 * m, C = 2 * M, R = Qrows + C;
    const int bs = 128;
    if (c->utilde) {
        k_proxy_box<<<dim3((M + 63) / 64, c->ncell), 64, 0, st>>>(M, c->cells, f.e2, f.yp, f.ypf);
        BIE_LAUNCH(c, "k_proxy_box");
    }
    k_build_Q<<<dim3((m * M + bs - 1) / bs, c->ncell), bs, 0, st>>>(f.A, R, m, M, c->gl_s, f.yp, c->cells, f.e2);
    BIE_LAUNCH(c, "k_build_Q");
    k_qr<<<c->ncell, 1024, 0, st>>>(f.A, R, C, Qrows, c->opts.lam_rel, f.beta);
    BIE_LAUNCH(c, "k_qr");
    k_form_P<<<dim3(Qrows, c->ncell), 256, R * sizeof(double), st>>>(f.A, R, C, f.beta, f.P);
    BIE_LAUNCH(c, "k_form_P");
    return build_wall_table(c, f.e2, f.wall, st);
}

int build_proxy_fit(bie_ctx* c) {
    ProxyFit f{c->A, c->beta, c->P, c->wall, c->e2d, c->yp, c->ypf};
    return build_proxy_fit_to(c, f, c->stream);
}

}  // namespace bie
