// GMRES (Sec. 6.2, remark on GMRES with the pressure fix) and the forward-
// Euler time step (Sec. 7).
//
// Krylov vectors live on the device (2N doubles each); orthogonalisation is
// classical Gram-Schmidt applied twice (CGS2) with deterministic block
// reductions.  The (k+2)-entry Hessenberg column is copied to the host, where
// the Givens rotations and the final triangular solve run (O(k^2) scalars).
//
// Batches: the cells of a context are independent systems.  They run in
// lockstep -- one operator application per iteration serves every cell --
// but each cell has its own Arnoldi process: the dot products are reduced per
// cell (the reduction chunks never straddle two cells), the coefficients of
// every vector update are per cell, and each cell has its own Hessenberg
// matrix and convergence test.  A converged cell is switched off: the near
// sums skip its work items and its Krylov vectors stay zero.
//
// BIE_MIXED: iterative refinement -- the residual r = b - A64 x uses the
// FP64-class operator; the correction solves A32 d = r by GMRES on the
// single-precision-pair operator to opts.inner_tol; x += d; repeat until
// ||r_c|| / ||b_c|| <= opts.gmres_tol in every cell c.  When a sweep meets
// its inner tolerance but cuts the FP64-class residual by less than
// kStallRatio, the remaining sweeps solve for d on the double-float operator
// to the final tolerance instead, and if those stall too the residual is
// taken with native FP64 pair sums.  BIE_FP64 / BIE_DF64:
// GMRES directly on the native-double / double-float operator.
#include <cmath>
#include <cstdio>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

constexpr double kStallRatio = 0.1;

__device__ inline double wsum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduction chunks of kDotChunk vector entries that never span two cells.
int build_dot_chunks(bie_ctx* c) {
    std::vector<int4> ch;
    std::vector<int2> cc(c->ncell);
    for (int ci = 0; ci < c->ncell; ++ci) {
        const Cell& cl = c->cells_h[ci];
        const int e0 = 2 * cl.node_off, e1 = 2 * (cl.node_off + cl.n_nodes);
        cc[ci] = make_int2((int)ch.size(), 0);
        for (int e = e0; e < e1; e += kDotChunk) ch.push_back(make_int4(ci, e, std::min(e1, e + kDotChunk), 0));
        cc[ci].y = (int)ch.size() - cc[ci].x;
    }
    c->sv.nchunks = (int)ch.size();
    BIE_CUDA(c, cudaMalloc((void**)&c->sv.chunks, ch.size() * sizeof(int4)));
    BIE_CUDA(c, cudaMalloc((void**)&c->sv.cell_chunks, cc.size() * sizeof(int2)));
    BIE_CUDA(c, cudaMalloc((void**)&c->sv.dpart, (size_t)(c->sv.kmax + 2 + kMaxAug) * ch.size() * sizeof(double)));
    BIE_CUDA(c, cudaMemcpy(c->sv.chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice));
    BIE_CUDA(c, cudaMemcpy(c->sv.cell_chunks, cc.data(), cc.size() * sizeof(int2), cudaMemcpyHostToDevice));
    return BIE_OK;
}

// Classical Gram-Schmidt building blocks for every cell at once.
// k_dots: block (b, g) writes the partial dot products V_j . w over reduction
// chunk b (kDotChunk entries of one cell) for the eight vectors j = 8g .. 8g+7
// (one warp each); V = w with nv = 1 gives the partial squared norms.  With a
// ticket, the last block to finish also forms the sums of k_fin (below) in
// the same fixed order, saving a launch when there are few of them.
template <int LG>
__device__ void fin_items(const double* __restrict__ part, int nchunks, int nv, const int2* __restrict__ cell_chunks,
                          int ncell, double* __restrict__ h, const Cell* __restrict__ cells, double* __restrict__ fac,
                          int gthread, int nthreads, bool bypass_l1) {
    // LG consecutive threads per (j, cell) item; every thread runs the same
    // number of rounds, so the shuffles see whole warps
    const int sub = gthread & (LG - 1);
    const int items = nv * ncell, groups = nthreads / LG;
    for (int r0 = 0; r0 < items; r0 += groups) {
        const int idx = r0 + gthread / LG;
        double s = 0;
        int cell = 0;
        if (idx < items) {
            const int j = idx / ncell;
            cell = idx - j * ncell;
            const int2 cc = cell_chunks[cell];
            const double* pp = part + (size_t)j * nchunks + cc.x;
#pragma unroll 4
            for (int b = sub; b < cc.y; b += LG) s += bypass_l1 ? __ldcg(pp + b) : pp[b];
        }
#pragma unroll
        for (int o = LG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (idx < items && sub == 0) {
            h[idx] = s;
            if (fac) fac[cell] = (cells[cell].active && s > 0) ? 1.0 / sqrt(s) : 0.0;
        }
    }
}

__global__ void __launch_bounds__(256)
k_dots(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ w,
       const int4* __restrict__ chunks, int nchunks, double* __restrict__ part, unsigned int* __restrict__ ticket,
       const int2* __restrict__ cell_chunks, int ncell, double* __restrict__ h, const Cell* __restrict__ cells,
       double* __restrict__ fac) {
    __shared__ bool last;
    const int j = blockIdx.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j < nv) {
        const int4 ch = chunks[blockIdx.x];
        const double* v = V + (size_t)j * ld;
        double s = 0;
        for (int i = ch.y + lane; i < ch.z; i += 32) s += v[i] * w[i];
        s = wsum(s);
        if (lane == 0) part[(size_t)j * nchunks + blockIdx.x] = s;
    }
    if (!ticket) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    fin_items<8>(part, nchunks, nv, cell_chunks, ncell, h, cells, fac, threadIdx.x, blockDim.x, true);
    if (threadIdx.x == 0) *ticket = 0u;
}

// One warp per (j, cell): h[j * ncell + cell] = the cell's chunk partials
// added in a fixed order.  With fac (squared norms, nv = 1) also the
// normalisation factor 1 / sqrt(h) of every active cell (0 for the others).
__global__ void k_fin(const double* __restrict__ part, int nchunks, int nv, const int2* __restrict__ cell_chunks,
                      int ncell, double* __restrict__ h, const Cell* __restrict__ cells, double* __restrict__ fac) {
    fin_items<32>(part, nchunks, nv, cell_chunks, ncell, h, cells, fac, blockIdx.x * blockDim.x + threadIdx.x,
                  gridDim.x * blockDim.x, false);
}

// w -= sum_j h[j * ncell + cell] V_j  (cell of each entry from node_cell);
// eight lanes per entry split the vectors and combine with shuffles (fixed
// order: deterministic), which keeps enough loads in flight for short vectors.
__global__ void __launch_bounds__(256)
k_update(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ h, int ncell,
         const int* __restrict__ node_cell, double* __restrict__ w, int n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int sub = (int)(t & 7);
    const int i0 = (int)(t >> 3);
    const int i = i0 < n ? i0 : n - 1;
    const double* hc = h + node_cell[i >> 1];
    double s = 0;
    for (int j = sub; j < nv; j += 8) s += hc[(size_t)j * ncell] * V[(size_t)j * ld + i];
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (sub == 0 && i0 < n) w[i] -= s;
}

// h = V^T w per cell (partials, then the fixed-order sums)
static int mdots(bie_ctx* c, const double* V, size_t ld, int nv, const double* w, double* h, double* fac) {
    // few sums: the last block of k_dots forms them; many (large batches): k_fin
    const bool fused = (long long)nv * c->ncell <= 512;
    k_dots<<<dim3(c->sv.nchunks, (nv + 7) / 8), 256, 0, c->stream>>>(
        V, ld, nv, w, c->sv.chunks, c->sv.nchunks, c->sv.dpart, fused ? c->sv.ticket : nullptr, c->sv.cell_chunks,
        c->ncell, h, c->cells, fac);
    BIE_LAUNCH(c, "k_dots");
    if (!fused) {
        k_fin<<<(nv * c->ncell * 32 + 255) / 256, 256, 0, c->stream>>>(c->sv.dpart, c->sv.nchunks, nv,
                                                                     c->sv.cell_chunks, c->ncell, h, c->cells, fac);
        BIE_LAUNCH(c, "k_fin");
    }
    return BIE_OK;
}

// dst = a[cell] src; a zero factor writes zeros (switched-off cells)
__global__ void k_scale_copy(const double* src, const double* __restrict__ a, const int* __restrict__ node_cell,
                             double* dst, int n) {  // src and dst may be the same vector
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = a[node_cell[i >> 1]];
    dst[i] = f == 0.0 ? 0.0 : f * src[i];
}

__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a * x[i];
}

// y = a - b
__global__ void k_sub(const double* a, const double* b, double* y, int n) {  // y may alias a or b
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a[i] - b[i];
}

// x += sum_j coef[j * ncell + cell] V_j
__global__ void k_combine(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ coef, int ncell,
                          const int* __restrict__ node_cell, double* __restrict__ x, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* cc = coef + node_cell[i >> 1];
    double s = x[i];
    for (int j = 0; j < nv; ++j) {
        const double a = cc[(size_t)j * ncell];
        if (a != 0.0) s += a * V[(size_t)j * ld + i];  // vectors past a cell's own dimension are not read
    }
    x[i] = s;
}

// node_cell of vector entry i is node_cell[i >> 1]; the kernels above index
// it that way, so the vectors' entries must be node-major (x, y interleaved).

// Per-cell 2-norms of v.
static int dnorms(bie_ctx* c, const double* v, std::vector<double>& out) {
    double* d = c->sv.fac + c->ncell;  // ncell scratch after the normalisation factors
    if (int rc = mdots(c, v, 0, 1, v, d, nullptr)) return rc;
    out.resize(c->ncell);
    BIE_CUDA(c, cudaMemcpyAsync(out.data(), d, c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    for (double& x : out) x = std::sqrt(x);
    return BIE_OK;
}

// Switch cells on or off for the near sums (uploads the table if it changed).
static int set_active(bie_ctx* c, const std::vector<char>& on) {
    bool changed = false;
    for (int k = 0; k < c->ncell; ++k)
        if (c->cells_h[k].active != (int)on[k]) {
            c->cells_h[k].active = on[k];
            changed = true;
        }
    return changed ? upload_cells(c, c->stream) : BIE_OK;
}

// Orthonormalise the nu augmentation directions per cell: C~ = A U~ with
// orthonormal columns (classical Gram-Schmidt twice, the same operations on U
// so that A U~ = C~ stays exact up to rounding).  A direction whose image is
// (numerically) in the span of the earlier ones, or zero, is dropped (scaled
// to zero).  Ct and Ut hold A U and U on entry.
// scratch of the augmentation set-up, after the normalisation factors and the
// per-cell norms: squared norms before / after projection, projection
// coefficients of the two passes over r and of the orthonormalisation
constexpr double kAugMinRatio = 1e-4;  // smallest kept |projected| / |original| of an augmentation image

static double* aug_scratch(bie_ctx* c, int slot) {
    const size_t nc = c->ncell;
    switch (slot) {
        case 0: return c->sv.fac + 2 * nc;                 // n0 (nc)
        case 1: return c->sv.fac + 3 * nc;                 // n1 (nc)
        case 2: return c->sv.fac + 4 * nc;                 // pass A (kMaxAug x nc)
        case 3: return c->sv.fac + (4 + kMaxAug) * nc;     // pass B
        default: return c->sv.fac + (4 + 2 * kMaxAug) * nc;  // orthonormalisation
    }
}

// f = 1 / |c| per cell from squared norms n0 (before) and n1 (after
// projection); 0 when the direction is zero or within a relative 1e-4 of the
// span of the earlier ones: normalising the small remainder would magnify
// the error of A U (single-precision pairs: ~1e-7 relative) past 1e-3 and
// break the relation A U~ = C~ the augmented cycle relies on
__global__ void k_aug_fac(const double* __restrict__ n0, const double* __restrict__ n1, double* __restrict__ f,
                          int nc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nc) return;
    const double a = n0[q], b = n1[q];
    f[q] = (isfinite(b) && b > 0 && b > kAugMinRatio * kAugMinRatio * a) ? 1.0 / sqrt(b) : 0.0;
}

// Direction i of (Ct, Ut) per cell: project out directions 0 .. i-1 of Ct
// (classical Gram-Schmidt twice, the same operations on Ut so that
// A Ut_i = Ct_i stays exact up to rounding), then scale both by 1 / |Ct_i|
// (k_aug_fac).  Scratch: n0, n1, f (ncell each), hq (i x ncell).
static int orthonormalise_dir(bie_ctx* c, double* Ct, double* Ut, int i, double* n0, double* n1, double* hq,
                              double* f) {
    const int n = 2 * c->N, nc = c->ncell;
    const size_t ld = (size_t)n;
    const int gu = (int)((8LL * n + 255) / 256), gs = (n + 255) / 256;
    double* ci = Ct + (size_t)i * ld;
    double* ui = Ut + (size_t)i * ld;
    if (int rc = mdots(c, ci, 0, 1, ci, n0, nullptr)) return rc;
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
        if (int rc = mdots(c, Ct, ld, i, ci, hq, nullptr)) return rc;
        k_update<<<gu, 256, 0, c->stream>>>(Ct, ld, i, hq, nc, c->node_cell, ci, n);
        BIE_LAUNCH(c, "k_update");
        k_update<<<gu, 256, 0, c->stream>>>(Ut, ld, i, hq, nc, c->node_cell, ui, n);
        BIE_LAUNCH(c, "k_update");
    }
    if (int rc = mdots(c, ci, 0, 1, ci, n1, nullptr)) return rc;
    k_aug_fac<<<(nc + 255) / 256, 256, 0, c->stream>>>(n0, n1, f, nc);
    BIE_LAUNCH(c, "k_aug_fac");
    k_scale_copy<<<gs, 256, 0, c->stream>>>(ci, f, c->node_cell, ci, n);
    BIE_LAUNCH(c, "k_scale_copy");
    k_scale_copy<<<gs, 256, 0, c->stream>>>(ui, f, c->node_cell, ui, n);
    BIE_LAUNCH(c, "k_scale_copy");
    return BIE_OK;
}

// Orthonormalise the nu augmentation directions per cell: C~ = A U~ with
// orthonormal columns.  A direction whose image is (numerically) in the span
// of the earlier ones, or zero, is dropped (scaled to zero).  Ct and Ut hold
// A U and U on entry.
static int orthonormalise_aug(bie_ctx* c, double* Ct, double* Ut, int nu) {
    for (int i = 0; i < nu; ++i)
        if (int rc = orthonormalise_dir(c, Ct, Ut, i, aug_scratch(c, 0), aug_scratch(c, 1), aug_scratch(c, 4),
                                        c->sv.fac))
            return rc;
    return BIE_OK;
}

// One GMRES cycle per cell on A_prec x = b from the current x (device),
// in lockstep.  r holds b - A x on entry with per-cell norms beta (cells with
// beta = 0 do not take part).  Cell k stops when its Arnoldi residual
// estimate is <= atol[k] or after kmax steps; its iteration count goes to
// it[k] and its estimate to est[k].  *n_apply counts operator applications.
//
// Augmentation (nu > 0 directions U, 2N each, the same for all cells): the
// correction is sought in span(U) + K_k(A', r'), with C~ = A U~ orthonormal,
// r' = r - C~ C~^T r and A' = (I - C~ C~^T) A (a fixed recycled space, as in
// GCRO).  C~ occupies the first nu columns of the basis, so the Gram-Schmidt
// passes project it out of every new vector (A V_k = C~ B_k + V_{k+1} H_k);
// with y the usual GMRES coefficients, the update is V y + U~ (C~^T r - B y)
// and the residual is the usual GMRES residual of the projected system.
// Directions that predict the solution well leave a small r'; directions
// that do not only cost their applications.
//
// Pipelining: iteration k+1 (operator application, CGS2, normalisation of
// the next basis vector with the norm computed on the device) is enqueued
// before the host waits for iteration k's Hessenberg column, so the host's
// Givens rotations and convergence test overlap the GPU's next iteration.
// When the last cell converges at iteration k, iteration k+1 has already
// run and is discarded; a cell that converges is switched off from
// iteration k+2 on.
static int gmres_cycle(bie_ctx* c, int prec, double* x, const double* r, const std::vector<double>& beta_in,
                       const std::vector<double>& atol, std::vector<int>& it, std::vector<double>& est,
                       int* n_apply, const double* U = nullptr, int nu = 0) {
    const int n = 2 * c->N, nc = c->ncell;
    const int bs = 256, gs = (n + bs - 1) / bs;
    const int kmax = c->sv.kmax;
    const size_t ld = (size_t)n;
    const size_t slot = (2 * (size_t)(kmax + 1 + kMaxAug) + 1) * nc;  // h1, h2, norm of one iteration
    double* V = c->sv.V;             // [C~ (nu) | Krylov vectors (kmax + 1) | U~ (nu)]
    double* Vk = V + (size_t)nu * ld;
    double* Ut = Vk + (size_t)(kmax + 1) * ld;
    double* w = c->sv.w;
    double* fac_d = c->sv.fac;
    double* coef = c->sv.h + 2 * slot;  // (kmax + kMaxAug) x nc combination coefficients
    std::vector<double> beta = beta_in;
    std::vector<double> acoef((size_t)nu * nc, 0.0);  // C~^T r, per direction and cell
    it.assign(nc, 0);
    est.assign(nc, 0.0);
    if (nu > 0) {
        std::vector<char> on0(nc, 0);
        for (int q = 0; q < nc; ++q) on0[q] = beta[q] > 0;
        if (int rc = set_active(c, on0)) return rc;
        for (int i = 0; i < nu; ++i) {
            BIE_CUDA(c, cudaMemcpyAsync(Ut + (size_t)i * ld, U + (size_t)i * ld, ld * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->stream));
            if (int rc = apply_device(c, Ut + (size_t)i * ld, V + (size_t)i * ld, prec)) return rc;
            ++*n_apply;
        }
        if (int rc = orthonormalise_aug(c, V, Ut, nu)) return rc;
        // r' = r - C~ (C~^T r), twice; the coefficients stay on the device
        // until the end of the cycle
        const int gu = (int)((8LL * n + 255) / 256);
        BIE_CUDA(c, cudaMemcpyAsync(w, r, ld * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        for (int pass = 0; pass < 2; ++pass) {
            double* hq = aug_scratch(c, 2 + pass);
            if (int rc = mdots(c, V, ld, nu, w, hq, nullptr)) return rc;
            k_update<<<gu, 256, 0, c->stream>>>(V, ld, nu, hq, nc, c->node_cell, w, n);
            BIE_LAUNCH(c, "k_update");
        }
        std::vector<double> b2;
        if (int rc = dnorms(c, w, b2)) return rc;  // (synchronises: the passes' coefficients are ready)
        std::vector<double> hh(2 * (size_t)nu * nc);
        BIE_CUDA(c, cudaMemcpy(hh.data(), aug_scratch(c, 2), (size_t)nu * nc * sizeof(double), cudaMemcpyDeviceToHost));
        BIE_CUDA(c, cudaMemcpy(hh.data() + (size_t)nu * nc, aug_scratch(c, 3), (size_t)nu * nc * sizeof(double),
                               cudaMemcpyDeviceToHost));
        for (size_t e = 0; e < (size_t)nu * nc; ++e) acoef[e] = hh[e] + hh[(size_t)nu * nc + e];
        for (int q = 0; q < nc; ++q) beta[q] = beta[q] > 0 ? b2[q] : 0.0;
        r = w;
    }
    std::vector<std::vector<double>> H(nc);  // packed columns: column k holds k + 1 entries
    std::vector<std::vector<double>> Bc(nc); // C~^T A v_k: nu entries per column
    std::vector<std::vector<double>> cs(nc), sn(nc), g(nc);
    std::vector<char> on(nc, 0);
    std::vector<double> fac(nc, 0.0), hcol(kmax + 2);
    int n_on = 0;
    for (int k = 0; k < nc; ++k) {
        if (beta[k] > atol[k] || (nu == 0 && beta[k] > 0)) {
            on[k] = 1;
            ++n_on;
            fac[k] = 1.0 / beta[k];
            g[k].assign(1, beta[k]);
        }
        est[k] = beta[k];
    }
    if (n_on) {
        if (int rc = set_active(c, on)) return rc;
        BIE_CUDA(c, cudaMemcpyAsync(fac_d, fac.data(), nc * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        k_scale_copy<<<gs, bs, 0, c->stream>>>(r, fac_d, c->node_cell, Vk, n);
        BIE_LAUNCH(c, "k_scale_copy");
    }
    // right preconditioning (opts.precond): the Krylov space is that of A M^-1
    const bool pc = c->pc.s > 0;
    // enqueue iteration k: w = A (M^-1) V_k, CGS2 against [C~, V_0 .. V_k],
    // V_{k+1} = w / |w| per cell, and the projections to the pinned host slot k % 2
    auto enqueue = [&](int k) -> int {
        if (pc) {
            if (int rc = precond_apply(c, Vk + (size_t)k * ld, c->pc.z)) return rc;
            if (int rc = apply_device(c, c->pc.z, w, prec)) return rc;
        } else if (int rc = apply_device(c, Vk + (size_t)k * ld, w, prec)) {
            return rc;
        }
        ++*n_apply;
        const int nv = nu + k + 1;
        double* hb = c->sv.h + (size_t)(k & 1) * slot;
        double* h1 = hb;
        double* h2 = hb + (size_t)nv * nc;
        double* hn = hb + 2 * (size_t)nv * nc;
        // CGS2: two projections, then the norm and the normalisation factor
        const int gu = (int)((8LL * n + 255) / 256);
        if (int rc = mdots(c, V, ld, nv, w, h1, nullptr)) return rc;
        k_update<<<gu, 256, 0, c->stream>>>(V, ld, nv, h1, nc, c->node_cell, w, n);
        BIE_LAUNCH(c, "k_update");
        if (int rc = mdots(c, V, ld, nv, w, h2, nullptr)) return rc;
        k_update<<<gu, 256, 0, c->stream>>>(V, ld, nv, h2, nc, c->node_cell, w, n);
        BIE_LAUNCH(c, "k_update");
        if (int rc = mdots(c, w, 0, 1, w, hn, fac_d)) return rc;
        k_scale_copy<<<gs, bs, 0, c->stream>>>(w, fac_d, c->node_cell, Vk + (size_t)(k + 1) * ld, n);
        BIE_LAUNCH(c, "k_scale_copy");
        BIE_CUDA(c, cudaMemcpyAsync(c->sv.pinned + (size_t)(k & 1) * slot, hb,
                                    (2 * (size_t)nv + 1) * nc * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
        BIE_CUDA(c, cudaEventRecord(c->sv.ev[k & 1], c->stream));
        return BIE_OK;
    };
    if (n_on)
        if (int rc = enqueue(0)) return rc;
    for (int k = 0; k < kmax && n_on > 0; ++k) {
        if (k + 1 < kmax)
            if (int rc = enqueue(k + 1)) return rc;
        BIE_CUDA(c, cudaEventSynchronize(c->sv.ev[k & 1]));
        const int nv = nu + k + 1;
        const double* hh = c->sv.pinned + (size_t)(k & 1) * slot;
        const double* hh2 = hh + (size_t)nv * nc;
        const double* hhn = hh + 2 * (size_t)nv * nc;
        bool switched = false;
        for (int q = 0; q < nc; ++q) {
            if (!on[q]) continue;
            for (int i = 0; i < nu; ++i) Bc[q].push_back(hh[(size_t)i * nc + q] + hh2[(size_t)i * nc + q]);
            for (int j = 0; j <= k; ++j)
                hcol[j] = hh[(size_t)(nu + j) * nc + q] + hh2[(size_t)(nu + j) * nc + q];
            const double hk1 = std::sqrt(hhn[q]);
            if (!std::isfinite(hk1)) return fail(c, BIE_ENUMERIC, "non-finite Krylov vector in GMRES");
            hcol[k + 1] = hk1;
            // Givens
            for (int j = 0; j < k; ++j) {
                const double a = cs[q][j] * hcol[j] + sn[q][j] * hcol[j + 1];
                hcol[j + 1] = -sn[q][j] * hcol[j] + cs[q][j] * hcol[j + 1];
                hcol[j] = a;
            }
            const double den = std::hypot(hcol[k], hcol[k + 1]);
            cs[q].push_back(hcol[k] / den);
            sn[q].push_back(hcol[k + 1] / den);
            hcol[k] = den;
            g[q].push_back(-sn[q][k] * g[q][k]);
            g[q][k] = cs[q][k] * g[q][k];
            H[q].insert(H[q].end(), hcol.begin(), hcol.begin() + k + 1);
            it[q] = k + 1;
            est[q] = std::fabs(g[q][k + 1]);
            if (est[q] <= atol[q] || hk1 == 0.0) {
                on[q] = 0;
                --n_on;
                switched = true;
            }
        }
        if (switched && n_on > 0)
            if (int rc = set_active(c, on)) return rc;
    }
    // per cell: back substitution with its own Krylov dimension; the
    // augmentation coefficients C~^T r - B y
    int kk = 0;
    for (int q = 0; q < nc; ++q) kk = std::max(kk, it[q]);
    std::vector<double> cf((size_t)kk * nc, 0.0), ca((size_t)nu * nc, 0.0);
    for (int q = 0; q < nc; ++q) {
        const int kq = it[q];
        // column j of H[q] starts at j (j + 1) / 2
        auto Hq = [&](int i, int j) { return H[q][(size_t)j * (j + 1) / 2 + i]; };
        std::vector<double> yv(kq);
        for (int i = kq - 1; i >= 0; --i) {
            double s = g[q][i];
            for (int j = i + 1; j < kq; ++j) s -= Hq(i, j) * yv[j];
            yv[i] = s / Hq(i, i);
        }
        for (int j = 0; j < kq; ++j) cf[(size_t)j * nc + q] = yv[j];
        for (int i = 0; i < nu; ++i) {
            double s = acoef[(size_t)i * nc + q];
            for (int j = 0; j < kq; ++j) s -= Bc[q][(size_t)j * nu + i] * yv[j];
            ca[(size_t)i * nc + q] = beta_in[q] > 0 ? s : 0.0;
        }
    }
    if (kk > 0) {
        BIE_CUDA(c, cudaMemcpyAsync(coef, cf.data(), cf.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (pc) {
            // x += M^-1 (V y)
            BIE_CUDA(c, cudaMemsetAsync(c->pc.t, 0, ld * sizeof(double), c->stream));
            k_combine<<<gs, bs, 0, c->stream>>>(Vk, ld, kk, coef, nc, c->node_cell, c->pc.t, n);
            BIE_LAUNCH(c, "k_combine");
            if (int rc = precond_apply(c, c->pc.t, c->pc.z)) return rc;
            k_axpy<<<gs, bs, 0, c->stream>>>(1.0, c->pc.z, x, n);
            BIE_LAUNCH(c, "k_axpy");
        } else {
            k_combine<<<gs, bs, 0, c->stream>>>(Vk, ld, kk, coef, nc, c->node_cell, x, n);
            BIE_LAUNCH(c, "k_combine");
        }
    }
    if (nu > 0) {
        double* coef2 = coef + (size_t)kmax * nc;
        BIE_CUDA(c, cudaMemcpyAsync(coef2, ca.data(), ca.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        k_combine<<<gs, bs, 0, c->stream>>>(Ut, ld, nu, coef2, nc, c->node_cell, x, n);
        BIE_LAUNCH(c, "k_combine");
    }
    return BIE_OK;
}

int solve_device(bie_ctx* c, const double* b, double* x, bool use_guess, bie_solve_info* info, const double* U,
                 int nu, bool recycle_second) {
    const int n = 2 * c->N, nc = c->ncell;
    const int bs = 256, gs = (n + bs - 1) / bs;
    bie_solve_info inf{};
    std::vector<bie_solve_info> ci(nc, bie_solve_info{});
    std::vector<char> all_on(nc, 1);
    int rc = set_active(c, all_on);
    if (rc) return rc;
    std::vector<double> bnorm;
    if ((rc = dnorms(c, b, bnorm))) return rc;
    for (double v : bnorm)
        if (!std::isfinite(v)) return fail(c, BIE_ENUMERIC, "non-finite right-hand side");
    if (!use_guess) BIE_CUDA(c, cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
    const double tol = c->opts.gmres_tol;
    const bool mixed = c->opts.precision == BIE_MIXED;
    const int max_outer = mixed ? c->opts.max_refine : 20;
    // operator of the plain (non-refined) solver: native double or double-float
    const int plain_prec = c->opts.precision == BIE_DF64 ? BIE_DF64 : BIE_FP64;
    // operator of the refinement sweeps: single-precision pairs, until a sweep
    // that met its inner tolerance fails to cut the FP64-class residual
    // tenfold (the single-precision operator is then too far from the FP64
    // one for this geometry's conditioning, e.g. bodies ~1e-5 apart); the
    // remaining sweeps run GMRES on the double-float operator to the final
    // tolerance.  If those stall the same way, the residual itself is at the
    // double-float operator's accuracy (its rounding of the large, cancelling
    // near-contact terms, ~1e-8 of the right-hand side at 1e-5 gaps): the
    // residual switches to native FP64.
    int inner_prec = BIE_MIXED;
    int res_prec = c->opts.residual;
    std::vector<double> rn_prev(nc, 0.0);
    std::vector<char> met(nc, 0);
    // cells still iterating: a zero right-hand side has the solution 0
    std::vector<char> todo(nc, 1);
    for (int q = 0; q < nc; ++q)
        if (bnorm[q] == 0.0) {
            todo[q] = 0;
            const Cell& cl = c->cells_h[q];
            BIE_CUDA(c, cudaMemsetAsync(x + 2 * (size_t)cl.node_off, 0, 2 * (size_t)cl.n_nodes * sizeof(double),
                                        c->stream));
        }
    std::vector<double> rn, beta(nc), atol(nc), est;
    std::vector<int> its;
    bool d2_pending = false, d2_written = false;
    for (int outer = 0; outer <= max_outer; ++outer) {
        bool any = false;
        for (char t : todo) any |= t != 0;
        if (!any) break;
        // FP64-class residual (native double, or double-float when mixed) of
        // the cells still iterating; from a zero start it is b itself
        const bool from_zero = outer == 0 && !use_guess;
        if ((rc = set_active(c, todo))) return rc;
        if (from_zero) {
            BIE_CUDA(c, cudaMemcpyAsync(c->sv.r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            rn = bnorm;
        } else {
            rc = apply_device(c, x, c->sv.r, mixed ? res_prec : plain_prec);
            if (rc) return rc;
            ++inf.applies64;
            k_sub<<<gs, bs, 0, c->stream>>>(b, c->sv.r, c->sv.r, n);
            BIE_LAUNCH(c, "k_sub");
            if ((rc = dnorms(c, c->sv.r, rn))) return rc;
        }
        bool left = false;
        for (int q = 0; q < nc; ++q) {
            beta[q] = 0.0;
            if (!todo[q]) continue;
            if (!std::isfinite(rn[q])) return fail(c, BIE_ENUMERIC, "non-finite residual");
            ci[q].rel_residual = rn[q] / bnorm[q];
            if (!from_zero) ++ci[q].applies64;
            if (ci[q].rel_residual <= tol) {
                todo[q] = 0;
                continue;
            }
            left = true;
            beta[q] = rn[q];
            if (mixed && met[q] && rn[q] > kStallRatio * rn_prev[q]) {
                if (inner_prec == BIE_MIXED) inner_prec = BIE_DF64;
                else res_prec = BIE_FP64;
            }
        }
        for (int q = 0; q < nc; ++q)
            if (beta[q] > 0.0)
                atol[q] = (mixed && inner_prec == BIE_MIXED)
                              ? std::max(c->opts.inner_tol * rn[q], 0.5 * tol * bnorm[q])
                              : 0.5 * tol * bnorm[q];
        if (!left || outer == max_outer) break;
        int napply = 0;
        if (mixed) {
            BIE_CUDA(c, cudaMemsetAsync(c->sv.d, 0, n * sizeof(double), c->stream));
            // the second sweep corrects the single-precision operator's error,
            // which changes little from one time step to the next: its last
            // correction is a search direction for this one
            const bool second = recycle_second && outer == 1 && inner_prec == BIE_MIXED;
            const double* Ua = from_zero ? U : ((second && c->sv.have_d2) ? c->sv.d2 : nullptr);
            const int na = from_zero ? nu : ((second && c->sv.have_d2) ? 1 : 0);
            rc = gmres_cycle(c, inner_prec, c->sv.d, c->sv.r, beta, atol, its, est, &napply, Ua, na);
            if (rc) return rc;
            for (int q = 0; q < nc; ++q) {
                met[q] = beta[q] > 0.0 && est[q] <= atol[q];
                rn_prev[q] = rn[q];
            }
            if (second) {
                // kept for the next solve if this solve's first sweep was itself
                // augmented (a start-up solve's correction is not representative)
                BIE_CUDA(c, cudaMemcpyAsync(c->sv.d2, c->sv.d, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                            c->stream));
                d2_pending = d2_written = true;
            }
            k_axpy<<<gs, bs, 0, c->stream>>>(1.0, c->sv.d, x, n);
            BIE_LAUNCH(c, "k_axpy");
            (inner_prec == BIE_MIXED ? inf.applies32 : inf.applies64) += napply;
        } else {
            rc = gmres_cycle(c, plain_prec, x, c->sv.r, beta, atol, its, est, &napply, from_zero ? U : nullptr,
                             from_zero ? nu : 0);
            if (rc) return rc;
            inf.applies64 += napply;
        }
        int kmax_it = 0;
        for (int q = 0; q < nc; ++q) {
            if (beta[q] == 0.0) continue;
            ci[q].iterations += its[q];
            ci[q].refinements += 1;
            if (mixed && inner_prec == BIE_MIXED) ci[q].applies32 += its[q];
            else ci[q].applies64 += its[q];
            kmax_it = std::max(kmax_it, its[q]);
        }
        inf.iterations += kmax_it;
        inf.refinements += 1;
    }
    if ((rc = set_active(c, all_on))) return rc;
    double worst = 0;
    int worst_cell = 0;
    for (int q = 0; q < nc; ++q)
        if (ci[q].rel_residual > worst) {
            worst = ci[q].rel_residual;
            worst_cell = q;
        }
    if (d2_written) c->sv.have_d2 = d2_pending && nu >= 2;
    inf.rel_residual = worst;
    c->sv.cell_info = ci;
    if (info) *info = inf;
    if (worst > tol) {
        char msg[200];
        if (nc > 1)
            snprintf(msg, sizeof msg,
                     "solver stopped above tolerance: relative residual %.3e in cell %d after %d sweeps, %d "
                     "iterations",
                     worst, worst_cell, ci[worst_cell].refinements, ci[worst_cell].iterations);
        else
            snprintf(msg, sizeof msg,
                     "solver stopped above tolerance: relative residual %.3e after %d sweeps, %d iterations", worst,
                     inf.refinements, inf.iterations);
        return fail(c, BIE_ENOCONV, msg);
    }
    return BIE_OK;
}

}  // namespace bie
