// Effective viscosity by contour deformation (Sec. 6.4, Eq. contourdef), for
// the doubled-cell periodizer (n_images 4).
//
// mu_eff is the shear force per unit shear through a contour C from L to R
// below every body (Eq. mueff is the special case C = D, valid only when no
// body meets D).  Split each curve into its quadrant pieces by lattice
// coordinates (s, t) about the cell centre and translate the pieces by
// -e1 (s >= 0) and -e2 (t >= 0): the translated curve Gamma~ carries the
// periodizer's near sum seen from x, x - e1, x - e2 and x - e1 - e2.  Gauss'
// law on the two cells below U then gives, with every evaluation at least
// half a cell from every source,
//   F = 2 W(D - e2) + 2 W(D - e1 - e2) + W(R - e2) - W(L - e1 - e2)
//       - sum_{t_j >= 0} q_j + int_D T(v, q),
//   W(wall) = int over the wall of the traction of Gamma~'s sources (normal
//   (0, 1) on the D walls, the outward normal of L on the L and R walls),
//   mu_eff = mu + F_1 / (gamma |e1|),
// int_D T(v, q) the proxy correction's traction on D.  Each wall integral is
// a kContourGL-point Gauss-Legendre rule.  The pieces and signs are those
// that reproduce the near sum (the printed Gamma~ names Gamma_1 in two of its
// four pieces).
#include <cmath>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

constexpr int kContourGL = 32;     // Gauss-Legendre points per wall
constexpr int kContourSplits = 8;  // source splits per wall point

// Wall w of the contour (0: D - e2, 1: D - e1 - e2, 2: R - e2, 3: L - e1 - e2):
// midpoint, direction, normal, coefficient.
__device__ inline void contour_wall(const Cell& cl, int w, double* mid, double* along, double* nrm, double* coef) {
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = cl.e2[0], e2y = cl.e2[1];
    double e1[2] = {e1x, e1y}, e2[2] = {e2x, e2y}, nl[2], nd[2];
    wall_normals(e1, e2, nl, nd);
    const double C0 = cl.C[0], C1 = cl.C[1];
    if (w == 0) {
        mid[0] = C0 - 1.5 * e2x; mid[1] = C1 - 1.5 * e2y;
    } else if (w == 1) {
        mid[0] = C0 - e1x - 1.5 * e2x; mid[1] = C1 - e1y - 1.5 * e2y;
    } else if (w == 2) {
        mid[0] = C0 + 0.5 * e1x - e2x; mid[1] = C1 + 0.5 * e1y - e2y;
    } else {
        mid[0] = C0 - 1.5 * e1x - e2x; mid[1] = C1 - 1.5 * e1y - e2y;
    }
    along[0] = w < 2 ? e1x : e2x;
    along[1] = w < 2 ? e1y : e2y;
    nrm[0] = w < 2 ? 0.0 : nl[0];
    nrm[1] = w < 2 ? 1.0 : nl[1];
    *coef = w < 2 ? 2.0 : (w == 2 ? 1.0 : -1.0);
}

// Block (wp, split, cell): wall point wp < 4 kContourGL (wall wp / kContourGL,
// Gauss-Legendre node wp % kContourGL) against the split's nodes moved to
// Gamma~; wp == 4 kContourGL sums q over the nodes with t >= 0.  The block's
// sums go to part[((cell * splits + split) * (4 kContourGL + 1) + wp) * 2].
__global__ void __launch_bounds__(256)
k_contour_walls(const Src64* __restrict__ src64, const Cell* __restrict__ cells, const double* __restrict__ gl,
                double* __restrict__ part) {
    __shared__ double red[2][8];
    const int wp = blockIdx.x, sp = blockIdx.y, nsp = gridDim.y, cidx = blockIdx.z;
    const Cell& cl = cells[cidx];
    const bool qsum = wp == 4 * kContourGL;
    double px = 0, py = 0, n0 = 0, n1 = 0;
    if (!qsum) {
        double mid[2], along[2], nrm[2], coef;
        contour_wall(cl, wp / kContourGL, mid, along, nrm, &coef);
        const double s = gl[wp % kContourGL];
        px = mid[0] + s * along[0];
        py = mid[1] + s * along[1];
        n0 = nrm[0];
        n1 = nrm[1];
    }
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = cl.e2[0], e2y = cl.e2[1];
    double tx = 0, ty = 0;
    const int per = (cl.n_nodes + nsp - 1) / nsp;
    const int j0 = cl.node_off + sp * per, j1 = min(cl.node_off + cl.n_nodes, j0 + per);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const Src64 q = src64[j];
        const double dx = q.x - cl.C[0], dy = q.y - cl.C[1];
        const double ls = cl.inv[0] * dx + cl.inv[1] * dy, lt = cl.inv[2] * dx + cl.inv[3] * dy;
        if (qsum) {
            if (lt >= 0) {
                tx += q.z;
                ty += q.w;
            }
            continue;
        }
        double yx = q.x, yy = q.y;
        if (ls >= 0) {
            yx -= e1x;
            yy -= e1y;
        }
        if (lt >= 0) {
            yx -= e2x;
            yy -= e2y;
        }
        const double rx = px - yx, ry = py - yy;
        const double r2 = rx * rx + ry * ry;
        const double cc = (rx * n0 + ry * n1) * (rx * q.z + ry * q.w) / (r2 * r2);
        tx += cc * rx;
        ty += cc * ry;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        tx += __shfl_xor_sync(0xffffffffu, tx, o);
        ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
    if (lane == 0) {
        red[0][warp] = tx;
        red[1][warp] = ty;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double t = 0;
        for (int k = 0; k < nw; ++k) t += red[threadIdx.x][k];
        const double scale = qsum ? 1.0 : -1.0 / kPi;
        part[(((size_t)cidx * nsp + sp) * (4 * kContourGL + 1) + wp) * 2 + threadIdx.x] = t * scale;
    }
}

// One CTA per cell: the fixed-order sums of the wall integrals, the q sum and
// the proxy correction's traction on D; mu_eff = mu + F_1 / (gamma |e1|).
__global__ void k_contour_fin(const double* __restrict__ part, int nsp, const double* __restrict__ gl,
                              const Cell* __restrict__ cells, const double* __restrict__ ypall,
                              const double* __restrict__ xiall, int M, double* __restrict__ out) {
    __shared__ double red[2][33];
    const int cidx = blockIdx.x;
    const Cell& cl = cells[cidx];
    const double* glw = gl + kContourGL;
    const int np = 4 * kContourGL + 1;
    double fx = 0, fy = 0;
    // one thread per wall point (and the q sum)
    for (int wp = threadIdx.x; wp < np; wp += blockDim.x) {
        double sx = 0, sy = 0;
        for (int s = 0; s < nsp; ++s) {
            const double* p = part + (((size_t)cidx * nsp + s) * np + wp) * 2;
            sx += p[0];
            sy += p[1];
        }
        if (wp == 4 * kContourGL) {
            fx -= sx;
            fy -= sy;
        } else {
            double mid[2], along[2], nrm[2], coef;
            contour_wall(cl, wp / kContourGL, mid, along, nrm, &coef);
            const double f = coef * glw[wp % kContourGL] * sqrt(along[0] * along[0] + along[1] * along[1]);
            fx += f * sx;
            fy += f * sy;
        }
    }
    // the proxy correction's traction on D, normal (0, 1)
    const double* yp = ypall + (size_t)cidx * 2 * M;
    const double* xi = xiall + (size_t)cidx * 2 * M;
    const double l1 = sqrt(cl.e1[0] * cl.e1[0] + cl.e1[1] * cl.e1[1]);
    for (int l = threadIdx.x; l < kContourGL; l += blockDim.x) {
        const double X = cl.C[0] - 0.5 * cl.e2[0] + gl[l] * cl.e1[0];
        const double Y = cl.C[1] - 0.5 * cl.e2[1] + gl[l] * cl.e1[1];
        double tx = 0, ty = 0;
        for (int p = 0; p < M; ++p) {
            const double rx = X - yp[2 * p], ry = Y - yp[2 * p + 1];
            const double r2 = rx * rx + ry * ry;
            const double cc = ry * (rx * xi[p] + ry * xi[M + p]) / (r2 * r2);
            tx += cc * rx;
            ty += cc * ry;
        }
        const double f = -glw[l] * l1 / kPi;
        fx += f * tx;
        fy += f * ty;
    }
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = fx;
        red[1][warp] = fy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double F = 0;
        for (int k = 0; k < nw; ++k) F += red[0][k];
        out[cidx] = cl.mu + F / (cl.gamma * l1);
    }
}

// Gauss-Legendre nodes on (-1/2, 1/2) (ascending) and weights summing to 1.
static void gauss_legendre_half_weights(int m, std::vector<double>& s, std::vector<double>& w) {
    gauss_legendre_half(m, s);
    w.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        const double z = 2.0 * s[i];
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= m; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double dp = m * (z * p1 - p0) / (z * z - 1.0);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // half of 2 / ((1 - z^2) P'(z)^2)
    }
}

int mu_eff_contour_device(bie_ctx* c, const double* sigma, double* mu_eff) {
    if (!c->utilde) return fail(c, BIE_EINVAL, "the contour-deformation mu_eff needs the doubled-cell periodizer (n_images 4)");
    if (!c->glc) {
        std::vector<double> s, w;
        gauss_legendre_half_weights(kContourGL, s, w);
        s.insert(s.end(), w.begin(), w.end());
        BIE_CUDA(c, cudaMalloc((void**)&c->glc, s.size() * sizeof(double)));
        BIE_CUDA(c, cudaMemcpy(c->glc, s.data(), s.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    const size_t np = 4 * kContourGL + 1;
    const size_t need = (size_t)c->ncell * kContourSplits * np * 2;
    if (c->contour_part_n < need) {
        if (c->contour_part) BIE_CUDA(c, cudaFree(c->contour_part));
        c->contour_part = nullptr;
        BIE_CUDA(c, cudaMalloc((void**)&c->contour_part, need * sizeof(double)));
        c->contour_part_n = need;
    }
    if (int rc = fp64_moments_and_xi(c, sigma)) return rc;
    k_contour_walls<<<dim3((unsigned)np, kContourSplits, c->ncell), 256, 0, c->stream>>>(c->ws.src64, c->cells, c->glc,
                                                                                      c->contour_part);
    BIE_LAUNCH(c, "k_contour_walls");
    k_contour_fin<<<c->ncell, 128, 0, c->stream>>>(c->contour_part, kContourSplits, c->glc, c->cells, c->yp, c->ws.xi,
                                                   c->M, mu_eff);
    BIE_LAUNCH(c, "k_contour_fin");
    return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" int bie_mu_eff_contour(bie_ctx* c, const double* sigma, double* mu_eff, int32_t on_device) {
    if (!c || !sigma || !mu_eff) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t n2 = 2 * (size_t)c->N;
    const double* din = sigma;
    double* dout = mu_eff;
    if (!on_device) {
        BIE_CUDA(c, cudaMemcpyAsync(c->ws.sigma, sigma, n2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        din = c->ws.sigma;
        dout = c->ws.out;
    }
    c->ws_x = nullptr;
    if (int rc = mu_eff_contour_device(c, din, dout)) return rc;
    if (!on_device)
        BIE_CUDA(c, cudaMemcpyAsync(mu_eff, c->ws.out, c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}
