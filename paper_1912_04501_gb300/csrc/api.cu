// C ABI entry points (include/bie.h): argument checking, device memory
// ownership, host <-> device staging, and the forward-Euler time loop.
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>

#include "bie_internal.cuh"

namespace bie {

int fail(bie_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_check(bie_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? BIE_ENOMEM : BIE_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
static int dalloc(bie_ctx* c, T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
    if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc");
    return BIE_OK;
}

static void free_all(bie_ctx* c) {
    if (c->aux) cudaStreamSynchronize(c->aux);  // nothing of an application left in flight
    free_graph(c);
    free_precond(c);
    void* ptrs[] = {c->cells, c->node_cell, c->body_cell, c->x, c->y, c->nx, c->ny, c->w, c->kap, c->owner, c->body,
                    c->tgt32, c->posdf, c->xw, c->yw, c->imc, c->bimg, c->ws.src32n, c->ws.src64u, c->next.yp,
                    c->next.ypf, c->glc, c->contour_part, c->bshape, c->near_ctr,
                    c->gl_s, c->A, c->beta, c->P, c->wall, c->e2d, c->next.A, c->next.beta, c->next.P,
                    c->next.wall, c->next.e2, c->yp, c->ypf, c->scal, c->ws.sigma, c->ws.out, c->ws.src64, c->ws.src32,
                    c->ws.srcdf, c->ws.bodyF, c->ws.part, c->ws.gpart, c->ws.gt, c->ws.dticket, c->sv.ticket, c->ws.xi, c->ws.xif, c->ws.T, c->ws.vpart, c->sv.V,
                    c->sv.w, c->sv.r, c->sv.x, c->sv.b, c->sv.d, c->sv.h, c->sv.fac, c->sv.dpart,
                    c->sv.chunks,
                    c->sv.cell_chunks, c->sv.sigma_prev, c->sv.sigma_prev2, c->sv.aug, c->sv.d2,
                    c->sv.feat, c->sv.pred, c->cl.dmin, c->cl.dmin_prev, c->cl.ddir, c->cl.slots, c->cl.count, c->cl.pair_base, c->cl.pairs,
                    c->cl.blk_off, c->cl.blocks, c->cl.blocks32, c->cl.flags, c->cl.dtab, c->cl.dtab_off,
                    c->cl.bkd, c->cl.bcot, c->cl.bary, c->near[0].items,
                    c->near[1].items, c->near[2].items};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto e : c->ev_pool)
        if (e) cudaEventDestroy(e);
    c->ev_pool.clear();
    if (c->next_done) cudaEventDestroy(c->next_done);
    if (c->aux_fork) cudaEventDestroy(c->aux_fork);
    if (c->aux_join) cudaEventDestroy(c->aux_join);
    for (auto e : c->sv.ev)
        if (e) cudaEventDestroy(e);
    if (c->sv.pinned) cudaFreeHost(c->sv.pinned);
    if (c->cells_pinned) cudaFreeHost(c->cells_pinned);
    if (c->cells_ev) cudaEventDestroy(c->cells_ev);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
}

// Lattice vectors, image shifts m e1 + n e2 (index (n + 1) * 3 + (m + 1)) and
// wall lengths of one cell.
void cell_set_lattice(Cell& cl, const double* e1, const double* e2) {
    for (int k = 0; k < 2; ++k) {
        cl.e1[k] = e1[k];
        cl.e2[k] = e2[k];
    }
    int idx = 0;
    for (int n = -1; n <= 1; ++n)
        for (int m = -1; m <= 1; ++m, ++idx) {
            cl.sx[idx] = m * e1[0] + n * e2[0];
            cl.sy[idx] = m * e1[1] + n * e2[1];
            cl.sxf[idx] = (float)cl.sx[idx];
            cl.syf[idx] = (float)cl.sy[idx];
            cl.sxl[idx] = (float)(cl.sx[idx] - (double)cl.sxf[idx]);
            cl.syl[idx] = (float)(cl.sy[idx] - (double)cl.syf[idx]);
        }
    cl.l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    cl.l2 = std::sqrt(e2[0] * e2[0] + e2[1] * e2[1]);
    const double det = e1[0] * e2[1] - e1[1] * e2[0];
    cl.inv[0] = e2[1] / det;
    cl.inv[1] = -e2[0] / det;
    cl.inv[2] = -e1[1] / det;
    cl.inv[3] = e1[0] / det;
}

// Stream-ordered upload of the host mirror of the cell table through a
// page-locked staging copy (asynchronous: the host does not wait for the
// stream).  The staging copy is rewritten only after the previous upload has
// left it.
int upload_cells(bie_ctx* c, cudaStream_t st) {
    BIE_CUDA(c, cudaEventSynchronize(c->cells_ev));
    std::memcpy(c->cells_pinned, c->cells_h.data(), c->cells_h.size() * sizeof(Cell));
    BIE_CUDA(c, cudaMemcpyAsync(c->cells, c->cells_pinned, c->cells_h.size() * sizeof(Cell), cudaMemcpyHostToDevice,
                                st));
    BIE_CUDA(c, cudaEventRecord(c->cells_ev, st));
    return BIE_OK;
}

// Lattice of Sec. 7 per cell: e1 = (L1, 0) fixed,
// e2(t) = (s0 + gamma t L2 - L1 round(.), L2), round half away from zero.
static void lattice_at(const bie_ctx* c, int cell, double t, double* e2) {
    const Cell& cl = c->cells_h[cell];
    const double L1 = cl.e1[0];
    double sx = c->e2_0[2 * cell] + cl.gamma * t * c->e2_0[2 * cell + 1];
    sx -= L1 * std::round(sx / L1);
    e2[0] = sx;
    e2[1] = c->e2_0[2 * cell + 1];
}

// out = a - b (vectors of n doubles)
__global__ void k_diff(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

// network output (predicted density change / (mu |gamma| dt), N x 2 floats)
// -> a density direction in the solver's units
__global__ void k_pred_to_density(const float* __restrict__ pred, const int* __restrict__ node_cell,
                                  const Cell* __restrict__ cells, int N, double dt, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Cell& cl = cells[node_cell[i]];
    const double s = cl.mu * fabs(cl.gamma) * dt;
    out[2 * i] = s * pred[2 * i];
    out[2 * i + 1] = s * pred[2 * i + 1];
}

// Keep the last two densities: sigma_prev2 <- sigma_prev <- x.
static int push_density(bie_ctx* c, const double* x) {
    const size_t n2 = 2 * (size_t)c->N;
    if (c->sv.have_prev)
        BIE_CUDA(c, cudaMemcpyAsync(c->sv.sigma_prev2, c->sv.sigma_prev, n2 * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
    c->sv.have_prev2 = c->sv.have_prev;
    BIE_CUDA(c, cudaMemcpyAsync(c->sv.sigma_prev, x, n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    c->sv.have_prev = true;
    return BIE_OK;
}

// The augmentation directions of the next solve (warm_start 2 and 3): the
// previous density, its change over the last step, and (2) the network's
// direction.  Returns their number.
static int prepare_aug(bie_ctx* c, double dt, int* nu) {
    *nu = 0;
    const int mode = c->opts.warm_start;
    // the previous density alone is a poor direction (its residual is
    // concentrated where bodies moved relative to each other and slows the
    // projected GMRES down): augment only once its last change is known too
    if ((mode != 2 && mode != 3) || !c->sv.have_prev || !c->sv.have_prev2) return BIE_OK;
    const size_t n2 = 2 * (size_t)c->N;
    double* U = c->sv.aug;
    BIE_CUDA(c, cudaMemcpyAsync(U, c->sv.sigma_prev, n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    k_diff<<<(int)((n2 + 255) / 256), 256, 0, c->stream>>>(c->sv.sigma_prev, c->sv.sigma_prev2, U + n2, (int)n2);
    BIE_LAUNCH(c, "k_diff");
    *nu = 2;
    if (mode == 2 && c->net) {
        if (int rc = features_device(c, c->sv.feat)) return rc;
        if (int rc = net_forward_async(c, c->net, c->sv.feat, c->N, c->sv.pred)) return rc;
        k_pred_to_density<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->sv.pred, c->node_cell, c->cells, c->N, dt,
                                                                      U + (size_t)(*nu) * n2);
        BIE_LAUNCH(c, "k_pred_to_density");
        ++*nu;
    }
    return BIE_OK;
}

// Move and rotate every body by (v, omega) dt and wrap its centroid into its
// cell: lattice coordinates about the cell centre into [-1/2, 1/2).
__global__ void k_euler(double* __restrict__ body, int nb, const int* __restrict__ body_cell,
                        const Cell* __restrict__ cells, const double* __restrict__ v, const double* __restrict__ om,
                        double dt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Cell& cl = cells[body_cell[b]];
    const double e1x = cl.e1[0], e1y = cl.e1[1], e2x = cl.e2[0], e2y = cl.e2[1];
    double* bd = body + 8 * b;
    double X = bd[2] + dt * v[2 * b], Y = bd[3] + dt * v[2 * b + 1];
    bd[4] += dt * om[b];
    double det = e1x * e2y - e1y * e2x;
    double px = X - cl.C[0], py = Y - cl.C[1];
    double a = (px * e2y - py * e2x) / det, bb = (e1x * py - e1y * px) / det;
    double sa = floor(a + 0.5), sb = floor(bb + 0.5);
    bd[2] = X - (sa * e1x + sb * e2x);
    bd[3] = Y - (sa * e1y + sb * e2y);
}

constexpr int kEventPairs = 1024;

int prof_begin(bie_ctx* c, int kind) {
    if (!c->prof) return BIE_OK;
    if (c->ev_used == kEventPairs) {
        int rc = prof_fold(c);
        if (rc) return rc;
    }
    if (c->ev_pool.empty()) {
        c->ev_pool.resize(2 * kEventPairs);
        c->ev_kind.resize(kEventPairs);
        for (auto& e : c->ev_pool) BIE_CUDA(c, cudaEventCreate(&e));
    }
    c->ev_kind[c->ev_used] = kind;
    BIE_CUDA(c, cudaEventRecord(c->ev_pool[2 * c->ev_used], c->stream));
    return BIE_OK;
}

int prof_end(bie_ctx* c) {
    if (!c->prof) return BIE_OK;
    BIE_CUDA(c, cudaEventRecord(c->ev_pool[2 * c->ev_used + 1], c->stream));
    ++c->ev_used;
    return BIE_OK;
}

int prof_fold(bie_ctx* c) {
    if (c->ev_used == 0) return BIE_OK;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < c->ev_used; ++k) {
        float ms = 0;
        BIE_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]));
        if (c->ev_kind[k] == 0) {
            c->prof_acc.near32_launches++;
            c->prof_acc.near32_ms += ms;
        } else if (c->ev_kind[k] == 1) {
            c->prof_acc.near64_launches++;
            c->prof_acc.near64_ms += ms;
        } else {
            c->prof_acc.neardf_launches++;
            c->prof_acc.neardf_ms += ms;
        }
    }
    c->ev_used = 0;
    return BIE_OK;
}

static int rebuild(bie_ctx* c) {
    int rc = build_geometry(c);
    if (rc) return rc;
    rc = build_proxy_fit(c);
    if (rc) return rc;
    rc = build_close(c);
    if (rc) return rc;
    return build_precond(c);
}

// The current lattices' e2 (host mirror) to the device array the proxy fits read.
static int upload_e2(bie_ctx* c, double* dst, const std::vector<double>& e2, cudaStream_t st) {
    BIE_CUDA(c, cudaMemcpyAsync(dst, e2.data(), e2.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    return BIE_OK;
}

static std::vector<double> current_e2(const bie_ctx* c) {
    std::vector<double> e2(2 * (size_t)c->ncell);
    for (int k = 0; k < c->ncell; ++k) {
        e2[2 * k] = c->cells_h[k].e2[0];
        e2[2 * k + 1] = c->cells_h[k].e2[1];
    }
    return e2;
}

static int check_opts(const bie_opts& o, std::string& why) {
    if (o.precision != BIE_FP64 && o.precision != BIE_MIXED && o.precision != BIE_DF64)
        why = "precision must be BIE_FP64, BIE_MIXED or BIE_DF64";
    else if (o.n_proxy < 4 || o.n_proxy > kMaxProxy) why = "n_proxy out of range";
    else if (o.n_coll < 2 || o.n_coll > kMaxColl) why = "n_coll out of range";
    else if (!(o.proxy_radius > 0) || !(o.lam_rel >= 0) || !(o.gmres_tol > 0) || !(o.inner_tol > 0))
        why = "non-positive tolerance or radius";
    else if (o.gmres_max < 1 || o.gmres_max > 1000 || o.max_refine < 1) why = "gmres_max / max_refine out of range";
    else if (o.residual != BIE_FP64 && o.residual != BIE_DF64) why = "residual must be BIE_FP64 or BIE_DF64";
    else if (o.warm_start < 0 || o.warm_start > 3) why = "warm_start must be 0, 1, 2 or 3";
    else if (!(o.close_factor >= 0) || o.close_factor > 100 || o.close_capacity < 0)
        why = "close_factor must be in [0, 100], close_capacity >= 0";
    else if ((o.autotune != 0 && o.autotune != 1) || (o.graph != 0 && o.graph != 1) ||
             (o.precond != 0 && o.precond != 1))
        why = "autotune, graph and precond must be 0 or 1";
    else if (o.n_images != 9 && o.n_images != 4) why = "n_images must be 9 or 4";
    else if (o.n_images == 4 && o.n_proxy % 4 != 0) why = "n_images 4 needs n_proxy a multiple of 4";
    else if (o.n_images == 4 && o.autotune) why = "the tile-shape autotuner times the 3 x 3 near sum (n_images 9)";
    else if (o.close_rule != 0 && o.close_rule != 1) why = "close_rule must be 0 or 1";
    else return 0;
    return 1;
}

}  // namespace bie

using namespace bie;

extern "C" {

void bie_default_opts(bie_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = BIE_MIXED;
    o->n_proxy = 48;
    o->proxy_radius = 1.5;
    o->n_coll = 24;
    o->lam_rel = 1e-8;
    o->gmres_tol = 1e-10;
    o->gmres_max = 200;
    o->inner_tol = 1e-5;
    o->max_refine = 8;
    o->warm_start = 3;
    o->min_gap = 0.0;
    o->device = 0;
    o->close_factor = 10.0;
    o->close_capacity = 0;
    o->residual = BIE_DF64;
    o->autotune = 0;
    o->graph = 0;
    o->precond = 0;
    o->n_images = 9;
    o->close_rule = 0;
}

int bie_init_batch(bie_ctx** out, int32_t n_cells, const bie_cell* cells, const bie_body* bodies,
                   const bie_opts* opts) {
    if (!out) return BIE_EINVAL;
    *out = nullptr;
    if (!cells || !bodies || n_cells <= 0 || n_cells > kMaxCells) return BIE_EINVAL;
    bie_ctx* c = new (std::nothrow) bie_ctx();
    if (!c) return BIE_ENOMEM;
    if (opts) c->opts = *opts;
    else bie_default_opts(&c->opts);
    auto bad = [&](const std::string& m) {
        c->err = m;
        delete c;
        return BIE_EINVAL;
    };
    const bie_opts& o = c->opts;
    {
        std::string why;
        if (check_opts(o, why)) return bad(why);
        if (o.precond && n_cells > 1) return bad("precond is for single-cell contexts");
    }
    c->device = o.device;
    c->utilde = o.n_images == 4;
    c->srcmul = c->utilde ? 4 : 1;
    c->ncell = n_cells;
    c->M = o.n_proxy;
    c->m = o.n_coll;
    c->cells_h.assign(n_cells, Cell{});
    c->e2_0.assign(2 * (size_t)n_cells, 0.0);
    long long N = 0, nb = 0;
    for (int k = 0; k < n_cells; ++k) {
        const bie_cell& in = cells[k];
        if (in.n_bodies <= 0) return bad("every cell needs at least one body");
        if (!(in.mu > 0) || !std::isfinite(in.gamma)) return bad("mu must be positive, gamma finite");
        const bie_lattice& lat = in.lattice;
        double det = lat.e1[0] * lat.e2[1] - lat.e1[1] * lat.e2[0];
        if (!(std::fabs(det) > 1e-12)) return bad("degenerate lattice");
        Cell& cl = c->cells_h[k];
        cell_set_lattice(cl, lat.e1, lat.e2);
        cl.C[0] = lat.center[0];
        cl.C[1] = lat.center[1];
        cl.mu = in.mu;
        cl.gamma = in.gamma;
        cl.active = 1;
        c->e2_0[2 * k] = lat.e2[0];
        c->e2_0[2 * k + 1] = lat.e2[1];
        cl.body_off = (int)nb;
        cl.n_bodies = in.n_bodies;
        cl.node_off = (int)N;
        for (int j = 0; j < in.n_bodies; ++j, ++nb) {
            const bie_body& bd = bodies[nb];
            if (bd.shape != 0 && bd.shape != 1) return bad("shape must be 0 (ellipse) or 1 (star)");
            if (bd.n_nodes < 8 || bd.n_nodes > kMaxBodyNodes || (bd.n_nodes & 1))
                return bad("n_nodes must be even, 8.." + std::to_string(kMaxBodyNodes));
            if (bd.shape == 0 && (!(bd.p[0] > 0) || !(bd.p[1] > 0))) return bad("ellipse semi-axes must be positive");
            if (bd.shape == 1 && (!(bd.p[0] > 0) || !(bd.p[1] >= 0 && bd.p[1] < 1) || !(bd.p[2] >= 1) ||
                                  bd.p[2] > 64 || bd.p[2] != std::floor(bd.p[2])))
                return bad("star: r0 > 0, 0 <= eps < 1 and an integer k in 1..64");
            if (!std::isfinite(bd.xc[0]) || !std::isfinite(bd.xc[1]) || !std::isfinite(bd.theta))
                return bad("non-finite body position");
            c->n_nodes.push_back(bd.n_nodes);
            c->offsets.push_back((int)N);
            for (int q = 0; q < 8; ++q) c->body_host.push_back(0.0);
            double* h = &c->body_host[8 * (size_t)nb];
            // ellipse: the semi-axes; star: its bounding radius twice (the
            // kernels that only need a size read max(h[0], h[1]))
            h[0] = bd.shape == 1 ? bd.p[0] * (1.0 + bd.p[1]) : bd.p[0];
            h[1] = bd.shape == 1 ? bd.p[0] * (1.0 + bd.p[1]) : bd.p[1];
            c->bshape_host.push_back(bd.shape);
            for (int q = 0; q < 3; ++q) c->bshape_host.push_back(bd.shape == 1 ? bd.p[q] : (q < 2 ? bd.p[q] : 0.0));
            h[2] = bd.xc[0];
            h[3] = bd.xc[1];
            h[4] = bd.theta;
            h[5] = bd.n_nodes;
            h[6] = (double)N;
            N += bd.n_nodes;
            if (N > (1 << 24)) return bad("too many nodes");
        }
        cl.n_nodes = (int)(N - cl.node_off);
    }
    c->N = (int)N;
    c->nb = (int)nb;
    c->offsets.push_back(c->N);

    auto cu = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) return cuda_check(c, e, what);
        return 0;
    };
    int rc;
    if ((rc = cu(cudaSetDevice(c->device), "cudaSetDevice"))) {
        delete c;
        return rc;
    }
    // the wave model of the near-sum work items sizes them for this device
    if ((rc = cu(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device),
                 "cudaDeviceGetAttribute")) || c->sms <= 0) {
        delete c;
        return rc ? rc : BIE_ECUDA;
    }
    const int n = c->N, M = c->M, m = c->m;
    const size_t nc = (size_t)n_cells, nbs = (size_t)c->nb;
    const int R = 8 * m + 2 * M, Cc = 2 * M;
    // near-sum splits for the partial buffer (the same rule fills the items below)
    const size_t part = near_part_bytes(c);
    c->sv.kmax = o.gmres_max;
    const int kk = c->sv.kmax;
    rc = 0;
    rc = rc ? rc : dalloc(c, &c->cells, nc);
    if (!rc) rc = cu(cudaMallocHost((void**)&c->cells_pinned, nc * sizeof(Cell)), "cudaMallocHost");
    if (!rc) rc = cu(cudaEventCreateWithFlags(&c->cells_ev, cudaEventDisableTiming), "cudaEventCreate");
    rc = rc ? rc : dalloc(c, &c->node_cell, n);
    rc = rc ? rc : dalloc(c, &c->body_cell, nbs);
    rc = rc ? rc : dalloc(c, &c->x, n);
    rc = rc ? rc : dalloc(c, &c->y, n);
    rc = rc ? rc : dalloc(c, &c->nx, n);
    rc = rc ? rc : dalloc(c, &c->ny, n);
    rc = rc ? rc : dalloc(c, &c->w, n);
    rc = rc ? rc : dalloc(c, &c->kap, n);
    rc = rc ? rc : dalloc(c, &c->owner, n);
    rc = rc ? rc : dalloc(c, &c->body, 8 * nbs);
    rc = rc ? rc : dalloc(c, &c->tgt32, n);
    rc = rc ? rc : dalloc(c, &c->posdf, n);
    rc = rc ? rc : dalloc(c, &c->xw, n);
    rc = rc ? rc : dalloc(c, &c->yw, n);
    rc = rc ? rc : dalloc(c, &c->imc, n);
    rc = rc ? rc : dalloc(c, &c->bimg, nbs);
    rc = rc ? rc : dalloc(c, &c->bshape, 4 * nbs);
    rc = rc ? rc : dalloc(c, &c->near_ctr, 1);
    rc = rc ? rc : dalloc(c, &c->gl_s, m);
    rc = rc ? rc : dalloc(c, &c->A, nc * R * Cc);
    rc = rc ? rc : dalloc(c, &c->beta, nc * 2 * Cc);
    rc = rc ? rc : dalloc(c, &c->P, nc * Cc * 8 * m);
    rc = rc ? rc : dalloc(c, &c->wall, nc * kWallStride * 2 * m);
    rc = rc ? rc : dalloc(c, &c->e2d, 2 * nc);
    rc = rc ? rc : dalloc(c, &c->next.A, nc * R * Cc);
    rc = rc ? rc : dalloc(c, &c->next.beta, nc * 2 * Cc);
    rc = rc ? rc : dalloc(c, &c->next.P, nc * Cc * 8 * m);
    rc = rc ? rc : dalloc(c, &c->next.wall, nc * kWallStride * 2 * m);
    rc = rc ? rc : dalloc(c, &c->next.e2, 2 * nc);
    if (!rc) rc = cu(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cu(cudaEventCreateWithFlags(&c->next_done, cudaEventDisableTiming), "cudaEventCreate");
    if (!rc) rc = cu(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cu(cudaEventCreateWithFlags(&c->aux_fork, cudaEventDisableTiming), "cudaEventCreate");
    if (!rc) rc = cu(cudaEventCreateWithFlags(&c->aux_join, cudaEventDisableTiming), "cudaEventCreate");
    rc = rc ? rc : dalloc(c, &c->yp, nc * 2 * M);
    rc = rc ? rc : dalloc(c, &c->ypf, nc * M);
    rc = rc ? rc : dalloc(c, &c->next.yp, nc * 2 * M);
    rc = rc ? rc : dalloc(c, &c->next.ypf, nc * M);
    rc = rc ? rc : dalloc(c, &c->scal, 3 * nbs + nc + 8);
    rc = rc ? rc : dalloc(c, &c->ws.sigma, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->ws.out, 2 * (size_t)n);
    const size_t nsrc = (size_t)n * c->srcmul;  // near-sum source records
    rc = rc ? rc : dalloc(c, &c->ws.src64, n);
    rc = rc ? rc : dalloc(c, &c->ws.src32, nsrc);
    rc = rc ? rc : dalloc(c, (char**)&c->ws.srcdf, nsrc * 32);
    if (c->utilde) {
        rc = rc ? rc : dalloc(c, &c->ws.src32n, n);
        rc = rc ? rc : dalloc(c, &c->ws.src64u, nsrc);
    }
    rc = rc ? rc : dalloc(c, &c->ws.bodyF, 3 * nbs);
    rc = rc ? rc : dalloc(c, (char**)&c->ws.part, part);
    rc = rc ? rc : dalloc(c, &c->ws.gpart, nc * kDiscSplits * 8 * m);
    rc = rc ? rc : dalloc(c, &c->ws.xi, nc * 2 * M);
    rc = rc ? rc : dalloc(c, &c->ws.xif, nc * 2 * M);
    rc = rc ? rc : dalloc(c, &c->ws.gt, nc * 8 * m);
    rc = rc ? rc : dalloc(c, &c->ws.dticket, nc * 2 * m);
    rc = rc ? rc : dalloc(c, &c->sv.ticket, 1);
    if (!rc) rc = cu(cudaMemset(c->ws.dticket, 0, nc * 2 * m * sizeof(unsigned int)), "cudaMemset");
    if (!rc) rc = cu(cudaMemset(c->sv.ticket, 0, sizeof(unsigned int)), "cudaMemset");
    rc = rc ? rc : dalloc(c, &c->ws.T, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->ws.vpart, nbs * kVelSplits * 3);
    rc = rc ? rc : dalloc(c, &c->sv.V, (size_t)(kk + 1 + 2 * kMaxAug) * 2 * n);
    rc = rc ? rc : dalloc(c, &c->sv.w, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.r, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.x, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.b, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.d, 2 * (size_t)n);
    {
        const size_t slot = (2 * (size_t)(kk + 1 + kMaxAug) + 1) * nc;
        rc = rc ? rc : dalloc(c, &c->sv.h, 2 * slot + (size_t)(kk + kMaxAug) * nc);
        rc = rc ? rc : dalloc(c, &c->sv.fac, (4 + 3 * (size_t)kMaxAug) * nc);
        if (!rc) rc = cu(cudaMallocHost((void**)&c->sv.pinned, 2 * slot * sizeof(double)), "cudaMallocHost");
        for (int e = 0; e < 2 && !rc; ++e)
            rc = cu(cudaEventCreateWithFlags(&c->sv.ev[e], cudaEventDisableTiming), "cudaEventCreate");
    }
    rc = rc ? rc : dalloc(c, &c->sv.sigma_prev, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.sigma_prev2, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.aug, (size_t)kMaxAug * 2 * n);
    rc = rc ? rc : dalloc(c, &c->sv.d2, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->sv.feat, (size_t)kNetFeatures * n);
    rc = rc ? rc : dalloc(c, &c->sv.pred, 2 * (size_t)n);
    rc = rc ? rc : dalloc(c, &c->cl.dmin, n);
    rc = rc ? rc : dalloc(c, &c->cl.dmin_prev, n);
    rc = rc ? rc : dalloc(c, &c->cl.ddir, n);
    // "no nearby curve" until the first close-pair detection (0x7f7f7f7f ~ 3.4e38)
    if (!rc) rc = cu(cudaMemset(c->cl.dmin, 0x7f, n * sizeof(float)), "cudaMemset");
    if (!rc) rc = cu(cudaMemset(c->cl.dmin_prev, 0x7f, n * sizeof(float)), "cudaMemset");
    if (!rc) rc = cu(cudaMemset(c->cl.ddir, 0, n * sizeof(float2)), "cudaMemset");
    {
        int maxn = 0;
        for (int v : c->n_nodes) maxn = std::max(maxn, v);
        // a given close_capacity is a hard limit; without one the block storage
        // starts at 1024 bodies' worth of pairs and grows with the geometry
        c->cl.grow = o.close_capacity <= 0;
        c->cl.cap_pairs = o.close_capacity > 0 ? o.close_capacity : n;
        c->cl.cap_doubles = (long long)(c->cl.grow ? std::min(c->cl.cap_pairs, 1024) : c->cl.cap_pairs) * 3 * maxn;
        rc = rc ? rc : dalloc(c, &c->cl.slots, (size_t)n * kCloseSlots);
        rc = rc ? rc : dalloc(c, &c->cl.count, n);
        rc = rc ? rc : dalloc(c, &c->cl.pair_base, (size_t)n + 1);
        rc = rc ? rc : dalloc(c, &c->cl.pairs, c->cl.cap_pairs);
        rc = rc ? rc : dalloc(c, &c->cl.blk_off, c->cl.cap_pairs);
        rc = rc ? rc : dalloc(c, &c->cl.blocks, (size_t)c->cl.cap_doubles);
        rc = rc ? rc : dalloc(c, &c->cl.blocks32, (size_t)c->cl.cap_doubles);
        rc = rc ? rc : dalloc(c, &c->cl.flags, 10);
        c->cl.rule = o.close_rule;
        if (o.close_rule == 1) {
            c->cl.cap_bary = 2 * (c->cl.cap_doubles / 3) + 2;
            rc = rc ? rc : dalloc(c, &c->cl.bkd, n);
            rc = rc ? rc : dalloc(c, &c->cl.bcot, n);
            rc = rc ? rc : dalloc(c, &c->cl.bary, (size_t)c->cl.cap_bary);
        }
    }
    c->ws.part_bytes = part;
    // zeroed once: a cell that the solver switches off keeps finite partials
    if (!rc) rc = cu(cudaMemset(c->ws.part, 0, part), "cudaMemset");
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    std::vector<int> owner(n), node_cell(n), body_cell(c->nb);
    for (int b = 0; b < c->nb; ++b)
        for (int k = c->offsets[b]; k < c->offsets[b + 1]; ++k) owner[k] = b;
    for (int k = 0; k < n_cells; ++k) {
        const Cell& cl = c->cells_h[k];
        for (int i = cl.node_off; i < cl.node_off + cl.n_nodes; ++i) node_cell[i] = k;
        for (int b = cl.body_off; b < cl.body_off + cl.n_bodies; ++b) body_cell[b] = k;
    }
    gauss_legendre_half(m, c->gl_host);
    std::vector<double> yp(nc * 2 * M);
    for (int k = 0; k < n_cells; ++k)
        for (int p = 0; p < M; ++p) {
            double a = 2.0 * kPi * p / M;
            yp[(size_t)k * 2 * M + 2 * p] = c->cells_h[k].C[0] + o.proxy_radius * std::cos(a);
            yp[(size_t)k * 2 * M + 2 * p + 1] = c->cells_h[k].C[1] + o.proxy_radius * std::sin(a);
        }
    auto up = [&](void* d, const void* h, size_t bytes) {
        return cu(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice), "cudaMemcpy");
    };
    rc = up(c->owner, owner.data(), n * sizeof(int));
    rc = rc ? rc : up(c->node_cell, node_cell.data(), n * sizeof(int));
    rc = rc ? rc : up(c->body_cell, body_cell.data(), c->nb * sizeof(int));
    rc = rc ? rc : up(c->body, c->body_host.data(), c->body_host.size() * sizeof(double));
    rc = rc ? rc : up(c->bshape, c->bshape_host.data(), c->bshape_host.size() * sizeof(double));
    rc = rc ? rc : up(c->gl_s, c->gl_host.data(), m * sizeof(double));
    // the 3 x 3 periodizer's proxy circle does not move with the lattice: both
    // fits hold it (the doubled cell's wall proxies are placed with each fit)
    rc = rc ? rc : up(c->yp, yp.data(), yp.size() * sizeof(double));
    rc = rc ? rc : up(c->next.yp, yp.data(), yp.size() * sizeof(double));
    {
        std::vector<float2> ypf(nc * M);
        for (int k = 0; k < n_cells; ++k)
            for (int p = 0; p < M; ++p)
                ypf[(size_t)k * M + p] = make_float2((float)(yp[(size_t)k * 2 * M + 2 * p] - c->cells_h[k].C[0]),
                                                     (float)(yp[(size_t)k * 2 * M + 2 * p + 1] - c->cells_h[k].C[1]));
        rc = rc ? rc : up(c->ypf, ypf.data(), ypf.size() * sizeof(float2));
        rc = rc ? rc : up(c->next.ypf, ypf.data(), ypf.size() * sizeof(float2));
    }
    rc = rc ? rc : up(c->e2d, c->e2_0.data(), c->e2_0.size() * sizeof(double));
    rc = rc ? rc : build_near_items(c);
    rc = rc ? rc : build_dot_chunks(c);
    rc = rc ? rc : build_dirichlet_tables(c, 64);
    rc = rc ? rc : rebuild(c);
    if (o.autotune) rc = rc ? rc : autotune_near32(c);
    rc = rc ? rc : cu(cudaStreamSynchronize(c->stream), "init sync");
    if (rc) {
        std::string e = c->err;
        free_all(c);
        delete c;
        (void)e;
        return rc;
    }
    c->sv.cell_info.assign(n_cells, bie_solve_info{});
    *out = c;
    return BIE_OK;
}

int bie_init(bie_ctx** out, const bie_lattice* lat, double mu, double gamma, int32_t n_bodies,
             const bie_body* bodies, const bie_opts* opts) {
    if (!out) return BIE_EINVAL;
    *out = nullptr;
    if (!lat || !bodies || n_bodies <= 0) return BIE_EINVAL;
    bie_cell cell;
    cell.lattice = *lat;
    cell.mu = mu;
    cell.gamma = gamma;
    cell.n_bodies = n_bodies;
    return bie_init_batch(out, 1, &cell, bodies, opts);
}

void bie_destroy(bie_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

const char* bie_last_error(const bie_ctx* c) { return c ? c->err.c_str() : "null context"; }

int bie_size(const bie_ctx* c, int32_t* n_nodes, int32_t* n_bodies) {
    if (!c) return BIE_EINVAL;
    if (n_nodes) *n_nodes = c->N;
    if (n_bodies) *n_bodies = c->nb;
    return BIE_OK;
}

int bie_cells(const bie_ctx* c, int32_t* n_cells, int32_t* node_offset, int32_t* body_offset,
              bie_solve_info* last_solve) {
    if (!c) return BIE_EINVAL;
    if (n_cells) *n_cells = c->ncell;
    for (int k = 0; k < c->ncell; ++k) {
        const Cell& cl = c->cells_h[k];
        if (node_offset) node_offset[k] = cl.node_off;
        if (body_offset) body_offset[k] = cl.body_off;
        if (last_solve) last_solve[k] = c->sv.cell_info[k];
    }
    if (node_offset) node_offset[c->ncell] = c->N;
    if (body_offset) body_offset[c->ncell] = c->nb;
    return BIE_OK;
}

int bie_set_stream(bie_ctx* c, void* stream) {
    if (!c) return BIE_EINVAL;
    c->stream = (cudaStream_t)stream;
    return BIE_OK;
}

static int copy_out(bie_ctx* c, double* dst, const double* dev, size_t count, int on_device) {
    if (!dst) return BIE_OK;
    BIE_CUDA(c, cudaMemcpyAsync(dst, dev, count * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    return BIE_OK;
}

int bie_nodes(bie_ctx* c, double* x, double* n, double* w, double* kappa, int32_t on_device) {
    if (!c) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t N = c->N;
    auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x) {
        BIE_CUDA(c, cudaMemcpy2DAsync(x, 2 * sizeof(double), c->x, sizeof(double), sizeof(double), N, kind, c->stream));
        BIE_CUDA(c, cudaMemcpy2DAsync(x + 1, 2 * sizeof(double), c->y, sizeof(double), sizeof(double), N, kind, c->stream));
    }
    if (n) {
        BIE_CUDA(c, cudaMemcpy2DAsync(n, 2 * sizeof(double), c->nx, sizeof(double), sizeof(double), N, kind, c->stream));
        BIE_CUDA(c, cudaMemcpy2DAsync(n + 1, 2 * sizeof(double), c->ny, sizeof(double), sizeof(double), N, kind, c->stream));
    }
    int rc = copy_out(c, w, c->w, N, on_device);
    if (rc) return rc;
    rc = copy_out(c, kappa, c->kap, N, on_device);
    if (rc) return rc;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_apply(bie_ctx* c, const double* sigma, double* out, int32_t precision, int32_t on_device) {
    if (!c || !sigma || !out) return BIE_EINVAL;
    if (precision != BIE_FP64 && precision != BIE_MIXED && precision != BIE_DF64)
        return fail(c, BIE_EINVAL, "bad precision");
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t n2 = 2 * (size_t)c->N;
    const double* din = sigma;
    double* dout = out;
    if (!on_device) {
        BIE_CUDA(c, cudaMemcpyAsync(c->ws.sigma, sigma, n2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        din = c->ws.sigma;
        dout = c->ws.out;
    }
    int rc = apply_device(c, din, dout, precision);
    if (rc) return rc;
    if (!on_device)
        BIE_CUDA(c, cudaMemcpyAsync(out, c->ws.out, n2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_rhs(bie_ctx* c, double* b, int32_t on_device) {
    if (!c || !b) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    int rc = rhs_device(c, on_device ? b : c->ws.out);
    if (rc) return rc;
    if (!on_device)
        BIE_CUDA(c, cudaMemcpyAsync(b, c->ws.out, 2 * (size_t)c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_solve(bie_ctx* c, const double* rhs, double* sigma, int32_t use_guess, int32_t on_device,
              bie_solve_info* info) {
    if (!c || !sigma) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t n2 = 2 * (size_t)c->N;
    auto kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int rc;
    if (rhs) BIE_CUDA(c, cudaMemcpyAsync(c->sv.b, rhs, n2 * sizeof(double), kind, c->stream));
    else if ((rc = rhs_device(c, c->sv.b))) return rc;
    if (use_guess) BIE_CUDA(c, cudaMemcpyAsync(c->sv.x, sigma, n2 * sizeof(double), kind, c->stream));
    int src = solve_device(c, c->sv.b, c->sv.x, use_guess != 0, info);
    if (src && src != BIE_ENOCONV) return src;
    BIE_CUDA(c, cudaMemcpyAsync(sigma, c->sv.x, n2 * sizeof(double),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if ((rc = push_density(c, c->sv.x))) return rc;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return src;
}

int bie_velocities(bie_ctx* c, const double* sigma, double* v, double* omega, double* mu_eff, int32_t on_device) {
    if (!c || !sigma) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t n2 = 2 * (size_t)c->N;
    const double* din = sigma;
    if (!on_device) {
        BIE_CUDA(c, cudaMemcpyAsync(c->ws.sigma, sigma, n2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        din = c->ws.sigma;
    }
    double* dv = c->scal;
    double* dom = c->scal + 2 * c->nb;
    double* dmu = c->scal + 3 * c->nb;
    int rc = velocities_device(c, din, dv, dom, dmu);
    if (rc) return rc;
    if ((rc = copy_out(c, v, dv, 2 * (size_t)c->nb, on_device))) return rc;
    if ((rc = copy_out(c, omega, dom, c->nb, on_device))) return rc;
    if ((rc = copy_out(c, mu_eff, dmu, c->ncell, on_device))) return rc;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_step(bie_ctx* c, double dt, int32_t n_steps, double* mu_eff_out, bie_solve_info* info) {
    if (!c || n_steps < 0 || !std::isfinite(dt)) return BIE_EINVAL;
    for (const Cell& cl : c->cells_h)
        if (cl.e1[1] != 0.0) return fail(c, BIE_EINVAL, "time stepping needs e1 = (L1, 0)");
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t n2 = 2 * (size_t)c->N;
    double* dv = c->scal;
    double* dom = c->scal + 2 * c->nb;
    double* dmu = c->scal + 3 * c->nb;
    std::vector<double> e2n(2 * (size_t)c->ncell);
    for (int s = 0; s < n_steps; ++s) {
        // the next step's lattices are known now: fit their proxies on the
        // side stream while this step solves (the fits only depend on e2(t + dt))
        for (int k = 0; k < c->ncell; ++k) lattice_at(c, k, c->t + dt, &e2n[2 * k]);
        BIE_CUDA(c, cudaEventRecord(c->next_done, c->stream));  // inputs of the fit are ready
        BIE_CUDA(c, cudaStreamWaitEvent(c->side, c->next_done, 0));
        if (int rc = upload_e2(c, c->next.e2, e2n, c->side)) return rc;
        if (int rc = build_proxy_fit_to(c, c->next, c->side)) return rc;
        BIE_CUDA(c, cudaEventRecord(c->next_done, c->side));
        int rc = rhs_device(c, c->sv.b);
        if (rc) return rc;
        bool guess = c->opts.warm_start == 1 && c->sv.have_prev;
        if (guess)
            BIE_CUDA(c, cudaMemcpyAsync(c->sv.x, c->sv.sigma_prev, n2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                        c->stream));
        int nu = 0;
        if ((rc = prepare_aug(c, dt, &nu))) return rc;
        bie_solve_info inf{};
        rc = solve_device(c, c->sv.b, c->sv.x, guess, &inf, nu ? c->sv.aug : nullptr, nu,
                          c->opts.warm_start == 2 || c->opts.warm_start == 3);
        if (info) *info = inf;
        if (rc) return rc;
        if ((rc = push_density(c, c->sv.x))) return rc;
        rc = velocities_device(c, c->sv.x, dv, dom, dmu, true);
        if (rc) return rc;
        if (mu_eff_out)
            BIE_CUDA(c, cudaMemcpyAsync(mu_eff_out + (size_t)s * c->ncell, dmu, c->ncell * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream));
        c->t += dt;
        c->sv.dt_prev = dt;
        for (int k = 0; k < c->ncell; ++k) {
            Cell& cl = c->cells_h[k];
            const double e1[2] = {cl.e1[0], cl.e1[1]};
            cell_set_lattice(cl, e1, &e2n[2 * k]);
        }
        if ((rc = upload_cells(c, c->stream))) return rc;
        k_euler<<<(c->nb + 127) / 128, 128, 0, c->stream>>>(c->body, c->nb, c->body_cell, c->cells, dv, dom, dt);
        BIE_LAUNCH(c, "k_euler");
        // adopt the prefetched proxy fits, then rebuild nodes and close pairs
        BIE_CUDA(c, cudaStreamWaitEvent(c->stream, c->next_done, 0));
        std::swap(c->A, c->next.A);
        std::swap(c->beta, c->next.beta);
        std::swap(c->P, c->next.P);
        std::swap(c->wall, c->next.wall);
        std::swap(c->e2d, c->next.e2);
        std::swap(c->yp, c->next.yp);
        std::swap(c->ypf, c->next.ypf);
        if ((rc = build_geometry(c))) return rc;
        std::swap(c->cl.dmin, c->cl.dmin_prev);
        c->cl.have_dprev = true;
        if ((rc = build_close(c))) return rc;
        if ((rc = build_precond(c))) return rc;
        if (c->opts.min_gap > 0 && c->cl.min_gap < c->opts.min_gap) {
            char msg[160];
            snprintf(msg, sizeof msg, "bodies closer than min_gap after the step to t = %.6g: gap %.3e < %.3e", c->t,
                     c->cl.min_gap, c->opts.min_gap);
            return fail(c, BIE_ECOLLIDE, msg);
        }
    }
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_get_state(bie_ctx* c, double* t, double* e2, double* xc, double* theta, double* sigma) {
    if (!c) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    std::vector<double> h(8 * (size_t)c->nb);
    BIE_CUDA(c, cudaMemcpyAsync(h.data(), c->body, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (sigma) {
        if (c->sv.have_prev)
            BIE_CUDA(c, cudaMemcpyAsync(sigma, c->sv.sigma_prev, 2 * (size_t)c->N * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->stream));
        else
            std::memset(sigma, 0, 2 * (size_t)c->N * sizeof(double));
    }
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    if (t) *t = c->t;
    if (e2)
        for (int k = 0; k < c->ncell; ++k) {
            e2[2 * k] = c->cells_h[k].e2[0];
            e2[2 * k + 1] = c->cells_h[k].e2[1];
        }
    for (int b = 0; b < c->nb; ++b) {
        if (xc) {
            xc[2 * b] = h[8 * b + 2];
            xc[2 * b + 1] = h[8 * b + 3];
        }
        if (theta) theta[b] = h[8 * b + 4];
    }
    return BIE_OK;
}

int bie_set_state(bie_ctx* c, double t, const double* e2, const double* xc, const double* theta,
                  const double* sigma) {
    if (!c || !e2 || !xc || !theta) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    std::vector<double> h(8 * (size_t)c->nb);
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    BIE_CUDA(c, cudaMemcpy(h.data(), c->body, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int b = 0; b < c->nb; ++b) {
        h[8 * b + 2] = xc[2 * b];
        h[8 * b + 3] = xc[2 * b + 1];
        h[8 * b + 4] = theta[b];
    }
    c->t = t;
    for (int k = 0; k < c->ncell; ++k) {
        Cell& cl = c->cells_h[k];
        const double e1[2] = {cl.e1[0], cl.e1[1]};
        cell_set_lattice(cl, e1, e2 + 2 * k);
    }
    int rc = upload_cells(c, c->stream);
    if (rc) return rc;
    rc = upload_e2(c, c->e2d, current_e2(c), c->stream);
    if (rc) return rc;
    BIE_CUDA(c, cudaMemcpyAsync(c->body, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (sigma) {
        BIE_CUDA(c, cudaMemcpyAsync(c->sv.sigma_prev, sigma, 2 * (size_t)c->N * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream));
        c->sv.have_prev = true;
    } else {
        c->sv.have_prev = false;
    }
    c->sv.have_prev2 = false;
    c->sv.have_d2 = false;
    c->cl.have_dprev = false;
    rc = rebuild(c);
    if (rc) return rc;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_get_history(bie_ctx* c, double* sigma_prev2, double* d2, double* dt_prev, int32_t* have) {
    if (!c) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const bool h1 = c->sv.have_prev && c->sv.have_prev2, h2 = c->sv.have_d2;
    if (have) *have = (h1 ? 1 : 0) | (h2 ? 2 : 0);
    if (dt_prev) *dt_prev = c->sv.dt_prev;
    const size_t bytes = 2 * (size_t)c->N * sizeof(double);
    if (sigma_prev2) {
        if (h1) BIE_CUDA(c, cudaMemcpyAsync(sigma_prev2, c->sv.sigma_prev2, bytes, cudaMemcpyDeviceToHost, c->stream));
        else std::memset(sigma_prev2, 0, bytes);
    }
    if (d2) {
        if (h2) BIE_CUDA(c, cudaMemcpyAsync(d2, c->sv.d2, bytes, cudaMemcpyDeviceToHost, c->stream));
        else std::memset(d2, 0, bytes);
    }
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_set_history(bie_ctx* c, const double* sigma_prev2, const double* d2, double dt_prev) {
    if (!c || !std::isfinite(dt_prev) || dt_prev < 0) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    const size_t bytes = 2 * (size_t)c->N * sizeof(double);
    c->sv.dt_prev = dt_prev;
    c->sv.have_prev2 = false;
    c->sv.have_d2 = false;
    if (sigma_prev2 && c->sv.have_prev) {
        BIE_CUDA(c, cudaMemcpyAsync(c->sv.sigma_prev2, sigma_prev2, bytes, cudaMemcpyHostToDevice, c->stream));
        c->sv.have_prev2 = true;
    }
    if (d2) {
        BIE_CUDA(c, cudaMemcpyAsync(c->sv.d2, d2, bytes, cudaMemcpyHostToDevice, c->stream));
        c->sv.have_d2 = true;
    }
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_set_warm_net(bie_ctx* c, const bie_net* net) {
    if (!c) return BIE_EINVAL;
    if (net && net_inputs(net) != kNetFeatures)
        return fail(c, BIE_EINVAL, "the warm-start network must take " + std::to_string(kNetFeatures) + " inputs");
    c->net = net;
    return BIE_OK;
}

int bie_features(bie_ctx* c, float* X, int32_t on_device) {
    if (!c || !X) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    int rc = features_device(c, on_device ? X : c->sv.feat);
    if (rc) return rc;
    if (!on_device)
        BIE_CUDA(c, cudaMemcpyAsync(X, c->sv.feat, (size_t)kNetFeatures * c->N * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->stream));
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_set_partition(bie_ctx* c, int32_t body_begin, int32_t body_end,
                      int (*exchange)(double* y, int64_t n2, void* user), void* user) {
    if (!c) return BIE_EINVAL;
    if (c->ncell != 1) return fail(c, BIE_EINVAL, "a target partition is for single-cell contexts");
    if (body_begin < 0 || body_end > c->nb || body_begin >= body_end)
        return fail(c, BIE_EINVAL, "body range out of bounds");
    const bool whole = body_begin == 0 && body_end == c->nb;
    if (!whole && !exchange) return fail(c, BIE_EINVAL, "a proper partition needs an exchange callback");
    BIE_CUDA(c, cudaSetDevice(c->device));
    c->shard.on = !whole;
    c->shard.b0 = body_begin;
    c->shard.b1 = body_end;
    c->shard.n0 = c->offsets[body_begin];
    c->shard.n1 = c->offsets[body_end];
    c->shard.exchange = whole ? nullptr : exchange;
    c->shard.user = whole ? nullptr : user;
    int rc = build_near_items(c);
    if (rc) return rc;
    BIE_CUDA(c, cudaStreamSynchronize(c->stream));
    return BIE_OK;
}

int bie_device_sms(const bie_ctx* c, int32_t* sms) {
    if (!c || !sms) return BIE_EINVAL;
    *sms = c->sms;
    return BIE_OK;
}

int bie_near_shape(bie_ctx* c, int32_t* shape, float* ms) {
    if (!c) return BIE_EINVAL;
    if (shape) *shape = c->shape32;
    if (ms)
        for (int k = 0; k < kNear32Shapes; ++k) ms[k] = c->tune_ms[k];
    return BIE_OK;
}

int bie_close_info(bie_ctx* c, int32_t* n_pairs, int32_t* under_resolved) {
    if (!c) return BIE_EINVAL;
    if (n_pairs) *n_pairs = c->cl.npairs;
    if (under_resolved) *under_resolved = c->cl.under_resolved;
    return BIE_OK;
}

int bie_profile(bie_ctx* c, int32_t enable) {
    if (!c) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    if (!enable && c->prof) {
        int rc = prof_fold(c);
        if (rc) return rc;
    }
    c->prof = enable != 0;
    return BIE_OK;
}

int bie_profile_read(bie_ctx* c, bie_profile_info* info) {
    if (!c || !info) return BIE_EINVAL;
    BIE_CUDA(c, cudaSetDevice(c->device));
    int rc = prof_fold(c);
    if (rc) return rc;
    *info = c->prof_acc;
    info->launches = c->launches;
    c->prof_acc = bie_profile_info{};
    c->launches = 0;
    return BIE_OK;
}

}  // extern "C"
