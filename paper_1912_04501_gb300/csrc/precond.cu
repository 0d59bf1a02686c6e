// Contact-block right preconditioner (opts.precond; no counterpart in the
// paper).  When two curves nearly touch, the operator's near-singular part is
// the interaction of the nodes around the contact: the targets within the
// close-evaluation zone of another curve (or of their own body's periodic
// image).  With S that node set, the preconditioner is
//     M = A_SS on S (the dense FP64 operator block: half the identity, the
//         near-image kernel with its on-curve diagonal, the close-evaluation
//         blocks and the rigid completion of Eq. BIEPerturbed2), and
//     M = I / 2 elsewhere (the second-kind operator's identity part),
// and GMRES solves A M^-1 y = b, sigma = M^-1 y.  The proxy correction and
// the pressure fix (smooth and rank one) are left out of M.  M^-1 is formed
// once per geometry by Gauss-Jordan elimination with partial pivoting.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

// Block (a, b) of A_SS, a, b < s: 2 x 2 entries of the operator from the
// density at node j = nodes[b] to the value at node i = nodes[a].
// Row-major augmented matrix [A_SS | I], leading dimension 2n (n = 2s).
__global__ void k_pc_assemble(const int* __restrict__ nodes, int s, const double* __restrict__ x,
                              const double* __restrict__ y, const double* __restrict__ nx,
                              const double* __restrict__ ny, const double* __restrict__ w,
                              const double* __restrict__ kap, const int* __restrict__ owner,
                              const double* __restrict__ body, const int* __restrict__ node_cell,
                              const Cell* __restrict__ cells, double* __restrict__ aug) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)s * s) return;
    const int a = (int)(t / s), bcol = (int)(t % s);
    const int i = nodes[a], j = nodes[bcol];
    const Cell& cl = cells[node_cell[i]];
    const double n0 = nx[i], n1 = ny[i], wj = w[j];
    double B00 = 0, B01 = 0, B10 = 0, B11 = 0;
    // near images: G^t(x_i, y_j + shift; n_i) w_j, shift 0 left out for i = j
    for (int im = 0; im < 9; ++im) {
        if (i == j && im == 4) continue;
        const double rx = x[i] - (x[j] + cl.sx[im]), ry = y[i] - (y[j] + cl.sy[im]);
        const double r2 = rx * rx + ry * ry;
        const double cc = -(rx * n0 + ry * n1) * wj / (kPi * r2 * r2);
        B00 += cc * rx * rx;
        B01 += cc * rx * ry;
        B11 += cc * ry * ry;
    }
    B10 = B01;
    if (i == j) {
        // one half of the identity and the on-curve diagonal -(kappa / 2 pi) tau tau^T w
        const double t0 = -n1, t1 = n0, g = -(kap[i] / (2.0 * kPi)) * wj;
        B00 += 0.5 + g * t0 * t0;
        B01 += g * t0 * t1;
        B10 += g * t1 * t0;
        B11 += 0.5 + g * t1 * t1;
    }
    if (owner[i] == owner[j]) {
        // rigid completion: F_b (w_j I) and (x_i - x^c)^perp tau_b, tau_b's
        // weight for node j being (x_j - x^c)^perp w_j
        const int bd = owner[i];
        const double xc = body[8 * bd + 2], yc = body[8 * bd + 3];
        const double pi0 = -(y[i] - yc), pi1 = x[i] - xc, pj0 = -(y[j] - yc), pj1 = x[j] - xc;
        B00 += wj * (1.0 + pi0 * pj0);
        B01 += wj * pi0 * pj1;
        B10 += wj * pi1 * pj0;
        B11 += wj * (1.0 + pi1 * pj1);
    }
    const long long n = 2LL * s, ld = 2 * n;
    double* r0 = aug + (2LL * a) * ld;
    double* r1 = r0 + ld;
    r0[2 * bcol] = B00;
    r0[2 * bcol + 1] = B01;
    r1[2 * bcol] = B10;
    r1[2 * bcol + 1] = B11;
    r0[n + 2 * bcol] = (a == bcol) ? 1.0 : 0.0;
    r0[n + 2 * bcol + 1] = 0.0;
    r1[n + 2 * bcol] = 0.0;
    r1[n + 2 * bcol + 1] = (a == bcol) ? 1.0 : 0.0;
}

// Close-evaluation blocks restricted to S: one warp per row node a (its
// pairs in order, the lanes over the source body's nodes; a warp owns its
// two rows, so no two threads add to one entry at once).
__global__ void k_pc_close(const int* __restrict__ nodes, int s, const int* __restrict__ pos,
                           const int* __restrict__ pair_base, const int4* __restrict__ pairs,
                           const long long* __restrict__ blk_off, const double* __restrict__ blocks,
                           const double* __restrict__ body, double* __restrict__ aug) {
    const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (a >= s) return;
    const int i = nodes[a];
    const long long ld = 4LL * s;
    double* r0 = aug + (2LL * a) * ld;
    double* r1 = r0 + ld;
    for (int p = pair_base[i]; p < pair_base[i + 1]; ++p) {
        const int b = pairs[p].y;
        const int nbn = (int)body[8 * b + 5], off = (int)body[8 * b + 6];
        const double* C = blocks + blk_off[p];
        for (int k = lane; k < nbn; k += 32) {
            const int col = pos[off + k];
            if (col < 0) continue;
            r0[2 * col] += C[3 * k];
            r0[2 * col + 1] += C[3 * k + 1];
            r1[2 * col] += C[3 * k + 1];
            r1[2 * col + 1] += C[3 * k + 2];
        }
    }
}

// Gauss-Jordan step k on [M | I] (n rows, leading dimension 2n), one CTA:
// pivot row = largest |M[i][k]|, i >= k (ties: the lowest index); swap it
// into row k; prow = row k / pivot over the active columns k .. 2n - 1; f =
// column k.  (Left of column k the rows k .. n - 1 are zero; the right half
// is dense once rows have been exchanged.)  A zero pivot sets *status (the
// block is then not used).
__global__ void __launch_bounds__(1024) k_gj_pivot(double* __restrict__ aug, int n, int k,
                                                   double* __restrict__ f, double* __restrict__ prow,
                                                   int* __restrict__ status) {
    __shared__ double sv[32];
    __shared__ int si[32];
    __shared__ int piv;
    const long long ld = 2LL * n;
    double best = -1.0;
    int bi = n;
    for (int r = k + threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(aug[r * ld + k]);
        if (v > best || (v == best && r < bi)) {
            best = v;
            bi = r;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sv[wid] = best;
        si[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = -1.0;
        int bx = n;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
            if (sv[q] > bv || (sv[q] == bv && si[q] < bx)) {
                bv = sv[q];
                bx = si[q];
            }
        piv = (bv > 0.0 && isfinite(bv)) ? bx : -1;
        if (piv < 0) *status = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) return;
    if (p != k)
        for (long long j = threadIdx.x; j < ld; j += blockDim.x) {
            const double t = aug[(long long)k * ld + j];
            aug[(long long)k * ld + j] = aug[(long long)p * ld + j];
            aug[(long long)p * ld + j] = t;
        }
    __syncthreads();
    const double inv = 1.0 / aug[(long long)k * ld + k];
    for (int j = k + threadIdx.x; j < 2 * n; j += blockDim.x) prow[j] = aug[(long long)k * ld + j] * inv;
    for (int r = threadIdx.x; r < n; r += blockDim.x) f[r] = aug[(long long)r * ld + k];
}

// Gauss-Jordan step k, elimination: row k = prow; other rows -= f[i] prow,
// over the active columns k .. 2n - 1 (the others do not change at step k).
__global__ void k_gj_elim(double* __restrict__ aug, int n, int k, const double* __restrict__ f,
                          const double* __restrict__ prow, const int* __restrict__ status) {
    if (*status) return;
    const int width = 2 * n - k;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * width) return;
    const int r = (int)(t / width), j = k + (int)(t % width);
    const long long ld = 2LL * n;
    if (r == k)
        aug[r * ld + j] = prow[j];
    else
        aug[r * ld + j] -= f[r] * prow[j];
}

// z = M^-1 v: 2 v outside S ...
__global__ void k_pc_scale(const double* __restrict__ v, const int* __restrict__ pos, double* __restrict__ z,
                           int n2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n2) return;
    if (pos[e >> 1] < 0) z[e] = 2.0 * v[e];
}

// ... and A_SS^-1 v_S on S: one warp per row of the inverse (the right half
// of the eliminated [M | I]).
__global__ void k_pc_inv(const double* __restrict__ aug, int s, const int* __restrict__ nodes,
                         const double* __restrict__ v, double* __restrict__ z) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int n = 2 * s;
    if (row >= n) return;
    const double* a = aug + (long long)row * 2 * n + n;
    double acc = 0.0;
    for (int col = lane; col < n; col += 32) acc = fma(a[col], v[2 * nodes[col >> 1] + (col & 1)], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[2 * nodes[row >> 1] + (row & 1)] = acc;
}

int precond_apply(bie_ctx* c, const double* v, double* z) {
    const int n2 = 2 * c->N, s = c->pc.s;
    k_pc_scale<<<(n2 + 255) / 256, 256, 0, c->stream>>>(v, c->pc.pos, z, n2);
    BIE_LAUNCH(c, "k_pc_scale");
    k_pc_inv<<<(2 * s * 32 + 255) / 256, 256, 0, c->stream>>>(c->pc.aug, s, c->pc.nodes, v, z);
    BIE_LAUNCH(c, "k_pc_inv");
    return BIE_OK;
}

// Select S from the close-pair detection (nodes with another curve within
// the zone), assemble [A_SS | I] and invert.  s > kPcMaxNodes keeps the
// kPcMaxNodes closest nodes.  A singular block (not expected: A_SS is a
// principal block of a second-kind operator) leaves the preconditioner off.
int build_precond(bie_ctx* c) {
    c->pc.s = 0;
    if (!c->opts.precond) return BIE_OK;
    const int N = c->N;
    std::vector<float> dmin(N);
    BIE_CUDA(c, cudaMemcpyAsync(dmin.data(), c->cl.dmin, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<int> sel;
    for (int i = 0; i < N; ++i)
        if (dmin[i] < 1e30f) sel.push_back(i);
    if (sel.empty()) return BIE_OK;
    if ((int)sel.size() > kPcMaxNodes) {
        std::stable_sort(sel.begin(), sel.end(), [&](int p, int q) { return dmin[p] < dmin[q]; });
        sel.resize(kPcMaxNodes);
        std::sort(sel.begin(), sel.end());
    }
    const int s = (int)sel.size(), n = 2 * s;
    std::vector<int> pos(N, -1);
    for (int a = 0; a < s; ++a) pos[sel[a]] = a;
    if (s > c->pc.cap) {
        for (void* p : {(void*)c->pc.nodes, (void*)c->pc.aug, (void*)c->pc.f, (void*)c->pc.prow})
            if (p) BIE_CUDA(c, cudaFree(p));
        c->pc.nodes = nullptr;
        c->pc.aug = c->pc.f = c->pc.prow = nullptr;
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.nodes, s * sizeof(int)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.aug, (size_t)n * 2 * n * sizeof(double)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.f, n * sizeof(double)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.prow, 2 * (size_t)n * sizeof(double)));
        c->pc.cap = s;
    }
    if (!c->pc.pos) {
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.pos, N * sizeof(int)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.status, sizeof(int)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.z, 2 * (size_t)N * sizeof(double)));
        BIE_CUDA(c, cudaMalloc((void**)&c->pc.t, 2 * (size_t)N * sizeof(double)));
    }
    BIE_CUDA(c, cudaMemcpyAsync(c->pc.nodes, sel.data(), s * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA(c, cudaMemcpyAsync(c->pc.pos, pos.data(), N * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    BIE_CUDA(c, cudaMemsetAsync(c->pc.status, 0, sizeof(int), c->stream));
    const long long ss = (long long)s * s;
    k_pc_assemble<<<(int)((ss + 255) / 256), 256, 0, c->stream>>>(c->pc.nodes, s, c->x, c->y, c->nx, c->ny, c->w,
                                                                 c->kap, c->owner, c->body, c->node_cell, c->cells,
                                                                 c->pc.aug);
    BIE_LAUNCH(c, "k_pc_assemble");
    if (c->cl.npairs > 0) {
        k_pc_close<<<(s * 32 + 255) / 256, 256, 0, c->stream>>>(c->pc.nodes, s, c->pc.pos, c->cl.pair_base,
                                                               c->cl.pairs, c->cl.blk_off, c->cl.blocks, c->body,
                                                               c->pc.aug);
        BIE_LAUNCH(c, "k_pc_close");
    }
    for (int k = 0; k < n; ++k) {
        const long long work = (long long)n * (2 * n - k);
        k_gj_pivot<<<1, 1024, 0, c->stream>>>(c->pc.aug, n, k, c->pc.f, c->pc.prow, c->pc.status);
        k_gj_elim<<<(int)((work + 255) / 256), 256, 0, c->stream>>>(c->pc.aug, n, k, c->pc.f, c->pc.prow,
                                                                     c->pc.status);
    }
    BIE_LAUNCH(c, "k_gj");
    c->launches += 2LL * n - 1;
    int status = 0;
    BIE_CUDA(c, cudaMemcpyAsync(&status, c->pc.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    if (!status) c->pc.s = s;
    return BIE_OK;
}

void free_precond(bie_ctx* c) {
    for (void* p : {(void*)c->pc.nodes, (void*)c->pc.aug, (void*)c->pc.f, (void*)c->pc.prow, (void*)c->pc.pos,
                    (void*)c->pc.status, (void*)c->pc.z, (void*)c->pc.t})
        if (p) cudaFree(p);
    c->pc = {};
}

}  // namespace bie
