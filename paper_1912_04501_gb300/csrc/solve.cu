// GMRES (Sec. 6.2, remark on GMRES with the pressure fix) and the forward-
// Euler time step (Sec. 7).
//
// Krylov vectors live on the device (2N doubles each); orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2) with deterministic block
// reductions.  The (k+2)-entry Hessenberg column is copied to the host, where
// the Givens rotations and the final triangular solve run (O(k^2) scalars).
//
// BIE_MIXED: iterative refinement -- the residual r = b - A64 x uses the
// double-precision operator; the correction solves A32 d = r by GMRES on the
// single-precision-pair operator to opts.inner_tol; x += d; repeat until
// ||r|| / ||b|| <= opts.gmres_tol.
#include <cmath>
#include <cstdio>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

__device__ inline double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Multi-vector dot products h[j] = V_j . w (j < nv) in two deterministic
// passes: block b of kDotChunks sums its slice of the vectors (one warp per
// vector j at a time), then k_mdot_fin adds the kDotChunks partials of each j.
constexpr int kDotChunks = 64;

__global__ void __launch_bounds__(256)
k_mdot_part(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ w, int n,
            double* __restrict__ part) {
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < nv; j += nw) {
        const double* v = V + (size_t)j * ld;
        double s = 0;
        for (int i = i0 + lane; i < i1; i += 32) s += v[i] * w[i];
        s = wsum(s);
        if (lane == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// one warp per vector j: lanes add the partials, then a shuffle tree
__global__ void k_mdot_fin(const double* __restrict__ part, int nchunk, int nv, double* __restrict__ h) {
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (j >= nv) return;
    double s = 0;
    for (int b = lane; b < nchunk; b += 32) s += part[(size_t)j * nchunk + b];
    s = wsum(s);
    if (lane == 0) h[j] = s;
}

static int mdot(bie_ctx* c, const double* V, size_t ld, int nv, const double* w, int n, double* h) {
    k_mdot_part<<<kDotChunks, 256, 0, c->stream>>>(V, ld, nv, w, n, c->sv.dpart);
    BIE_LAUNCH(c, "k_mdot_part");
    k_mdot_fin<<<(nv * 32 + 255) / 256, 256, 0, c->stream>>>(c->sv.dpart, kDotChunks, nv, h);
    BIE_LAUNCH(c, "k_mdot_fin");
    return BIE_OK;
}

// w -= sum_j h[j] V_j
__global__ void k_mupdate(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ h,
                          double* __restrict__ w, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s0 = w[i], s1 = 0, s2 = 0, s3 = 0;
    int j = 0;
    for (; j + 4 <= nv; j += 4) {
        s0 -= h[j] * V[(size_t)j * ld + i];
        s1 -= h[j + 1] * V[(size_t)(j + 1) * ld + i];
        s2 -= h[j + 2] * V[(size_t)(j + 2) * ld + i];
        s3 -= h[j + 3] * V[(size_t)(j + 3) * ld + i];
    }
    for (; j < nv; ++j) s0 -= h[j] * V[(size_t)j * ld + i];
    w[i] = (s0 + s1) + (s2 + s3);
}

__global__ void k_scale_copy(const double* __restrict__ src, double a, double* __restrict__ dst, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = a * src[i];
}

__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

// y = a - b
__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] - b[i];
}

// x += sum_j c[j] V_j  (c on device)
__global__ void k_combine(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ c,
                          double* __restrict__ x, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = x[i];
    for (int j = 0; j < nv; ++j) s += c[j] * V[(size_t)j * ld + i];
    x[i] = s;
}

static int dnorm(bie_ctx* c, const double* v, int n, double* out) {
    if (int rc = mdot(c, v, 0, 1, v, n, c->sv.red)) return rc;
    double h;
    BIE_CUDA(c, cudaMemcpyAsync(&h, c->sv.red, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    *out = std::sqrt(h);
    return BIE_OK;
}

// One GMRES cycle on A_prec x = b from the current x (device), stopping when
// the Arnoldi residual estimate is <= atol or after kmax steps.  r must hold
// b - A x on entry, with norm beta.  Returns iterations in *it.
static int gmres_cycle(bie_ctx* c, int prec, double* x, const double* r, double beta, double atol, int* it,
                       double* est, int* n_apply) {
    const int n = 2 * c->N;
    const int bs = 256, gs = (n + bs - 1) / bs;
    const int gs64 = (n + 63) / 64;
    const int kmax = c->sv.kmax;
    const size_t ld = (size_t)n;
    double* V = c->sv.V;
    std::vector<double> H((size_t)(kmax + 1) * kmax, 0.0), cs(kmax), sn(kmax), g(kmax + 1, 0.0);
    std::vector<double> hcol(kmax + 2);
    g[0] = beta;
    k_scale_copy<<<gs, bs, 0, c->stream>>>(r, 1.0 / beta, V, n);
    BIE_LAUNCH(c, "k_scale_copy");
    int k = 0;
    double res = beta;
    for (k = 0; k < kmax; ++k) {
        double* w = c->sv.w;
        int rc = apply_device(c, V + (size_t)k * ld, w, prec);
        if (rc) return rc;
        ++*n_apply;
        // CGS2
        double* h1 = c->sv.h;
        double* h2 = c->sv.h + (kmax + 2);
        if ((rc = mdot(c, V, ld, k + 1, w, n, h1))) return rc;
        k_mupdate<<<gs64, 64, 0, c->stream>>>(V, ld, k + 1, h1, w, n);
        BIE_LAUNCH(c, "k_mupdate");
        if ((rc = mdot(c, V, ld, k + 1, w, n, h2))) return rc;
        k_mupdate<<<gs64, 64, 0, c->stream>>>(V, ld, k + 1, h2, w, n);
        BIE_LAUNCH(c, "k_mupdate");
        if ((rc = mdot(c, w, 0, 1, w, n, h2 + (kmax + 2)))) return rc;
        std::vector<double> hh(2 * (kmax + 2) + 1);
        BIE_CUDA(c, cudaMemcpyAsync(hh.data(), h1, (2 * (kmax + 2) + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
        BIE_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int j = 0; j <= k; ++j) hcol[j] = hh[j] + hh[(kmax + 2) + j];
        double hk1 = std::sqrt(hh[2 * (kmax + 2)]);
        if (!std::isfinite(hk1)) return fail(c, BIE_ENUMERIC, "non-finite Krylov vector in GMRES");
        hcol[k + 1] = hk1;
        if (hk1 > 0) {
            k_scale_copy<<<gs, bs, 0, c->stream>>>(w, 1.0 / hk1, V + (size_t)(k + 1) * ld, n);
            BIE_LAUNCH(c, "k_scale_copy");
        }
        // Givens
        for (int j = 0; j < k; ++j) {
            double a = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
            hcol[j + 1] = -sn[j] * hcol[j] + cs[j] * hcol[j + 1];
            hcol[j] = a;
        }
        double den = std::hypot(hcol[k], hcol[k + 1]);
        cs[k] = hcol[k] / den;
        sn[k] = hcol[k + 1] / den;
        hcol[k] = den;
        hcol[k + 1] = 0.0;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        for (int j = 0; j <= k; ++j) H[(size_t)j * kmax + k] = hcol[j];
        res = std::fabs(g[k + 1]);
        if (res <= atol || hk1 == 0.0) {
            ++k;
            break;
        }
    }
    int kk = std::min(k, kmax);
    std::vector<double> yv(kk);
    for (int i = kk - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < kk; ++j) s -= H[(size_t)i * kmax + j] * yv[j];
        yv[i] = s / H[(size_t)i * kmax + i];
    }
    BIE_CUDA(c, cudaMemcpyAsync(c->sv.h, yv.data(), kk * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    k_combine<<<gs, bs, 0, c->stream>>>(V, ld, kk, c->sv.h, x, n);
    BIE_LAUNCH(c, "k_combine");
    *it = kk;
    *est = res;
    return BIE_OK;
}

int solve_device(bie_ctx* c, const double* b, double* x, bool use_guess, bie_solve_info* info) {
    const int n = 2 * c->N;
    const int bs = 256, gs = (n + bs - 1) / bs;
    bie_solve_info inf{};
    double bnorm;
    int rc = dnorm(c, b, n, &bnorm);
    if (rc) return rc;
    if (!std::isfinite(bnorm)) return fail(c, BIE_ENUMERIC, "non-finite right-hand side");
    if (bnorm == 0.0) {
        BIE_CUDA(c, cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
        if (info) *info = inf;
        return BIE_OK;
    }
    if (!use_guess) BIE_CUDA(c, cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
    const double tol = c->opts.gmres_tol;
    const bool mixed = c->opts.precision == BIE_MIXED;
    const int max_outer = mixed ? c->opts.max_refine : 20;
    double rel = 0;
    for (int outer = 0; outer <= max_outer; ++outer) {
        // FP64-class residual (native double, or double-float when mixed)
        rc = apply_device(c, x, c->sv.r, mixed ? c->opts.residual : BIE_FP64);
        if (rc) return rc;
        ++inf.applies64;
        k_sub<<<gs, bs, 0, c->stream>>>(b, c->sv.r, c->sv.r, n);
        BIE_LAUNCH(c, "k_sub");
        double rn;
        rc = dnorm(c, c->sv.r, n, &rn);
        if (rc) return rc;
        if (!std::isfinite(rn)) return fail(c, BIE_ENUMERIC, "non-finite residual");
        rel = rn / bnorm;
        if (rel <= tol || outer == max_outer) break;
        int it = 0, napply = 0;
        double est;
        if (mixed) {
            BIE_CUDA(c, cudaMemsetAsync(c->sv.d, 0, n * sizeof(double), c->stream));
            double atol = std::max(c->opts.inner_tol * rn, 0.5 * tol * bnorm);
            rc = gmres_cycle(c, BIE_MIXED, c->sv.d, c->sv.r, rn, atol, &it, &est, &napply);
            if (rc) return rc;
            k_axpy<<<gs, bs, 0, c->stream>>>(1.0, c->sv.d, x, n);
            BIE_LAUNCH(c, "k_axpy");
            inf.applies32 += napply;
        } else {
            rc = gmres_cycle(c, BIE_FP64, x, c->sv.r, rn, 0.5 * tol * bnorm, &it, &est, &napply);
            if (rc) return rc;
            inf.applies64 += napply;
        }
        inf.iterations += it;
        inf.refinements += 1;
    }
    inf.rel_residual = rel;
    if (info) *info = inf;
    if (rel > tol) {
        char msg[160];
        snprintf(msg, sizeof msg, "solver stopped above tolerance: relative residual %.3e after %d sweeps, %d iterations",
                 rel, inf.refinements, inf.iterations);
        return fail(c, BIE_ENOCONV, msg);
    }
    return BIE_OK;
}

}  // namespace bie
