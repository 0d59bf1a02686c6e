// Internal declarations of the GB300 periodized Stokes BIE library.
//
// A context holds one or more independent unit cells (a batch); a single cell
// is a batch of one.  Nodes and bodies of all cells are concatenated; every
// kernel finds a node's or body's cell through node_cell / body_cell and the
// per-cell table `cells`.
//
// Layout in HBM (all device arrays owned by the context):
//   geometry  : x, y, nx, ny, w, kappa (N doubles each, SoA), owner (N ints, global
//               body index), node_cell (N), body (nb x 8 doubles: a, b, xc, yc, theta,
//               n, node offset, h), body_cell (nb), tgt32 (N float4: x - C, y - C, nx, ny),
//               posdf (N float4: x - C, y - C as double-float pairs)
//   densities : 2N doubles, node-major (x, y interleaved) == double2[N]
//   sources   : src32 (N float4: x - C, y - C, qx, qy), src64 (N Src64: x, y, qx, qy),
//               srcdf (N double-float records)
//   per cell  : Cell table; proxies yp (M x 2), stacked [Q; lam I] (column-major,
//               R = 8m + 2M rows, 2M cols), Householder scalars, P (2M x 8m, row-major),
//               wall table (2m x 16), proxy strengths xi (2M), discrepancy partials
//   near sums : work items (cell, target tile, source split) per precision; partial
//               sums per cell: splits x N_cell (float2 or double2)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bie.h"

namespace bie {

constexpr double kPi = 3.14159265358979323846;
#ifndef BIE_NEAR_THREADS
#define BIE_NEAR_THREADS 128
#endif
constexpr int kNearThreads = BIE_NEAR_THREADS;  // threads per near-sum block
constexpr int kNearTile = 256;                  // sources staged per shared-memory tile
// Tile shapes of the single-precision near sum: packed (two images per f32x2
// instruction) or scalar, targets per thread, and the resident CTAs per SM
// the kernel is compiled for (its register budget; also the wave model's
// slots).  Measured on GB300, the first (packed, 2 targets per thread, 5 CTAs
// per SM) beats the best scalar shape (3 targets per thread) by 1 % on the
// 25-ellipse cell, 4 % on the 400-ellipse cell and 9 % on the 64-cell
// ensemble, so it is the default; opts.autotune times all of them on the
// context's own cells and keeps the fastest.
struct Near32Shape {
    int packed, tpt, ctas;
};
constexpr int kNear32Shapes = 5;
// the default shape (entry 0) can be rebuilt with other values for measurement
#ifndef BIE_NEAR32_TPT
#define BIE_NEAR32_TPT 2
#endif
#ifndef BIE_NEAR32_CTAS
#define BIE_NEAR32_CTAS 5
#endif
constexpr Near32Shape kNear32ShapeList[kNear32Shapes] = {
    {1, BIE_NEAR32_TPT, BIE_NEAR32_CTAS}, {1, 1, 8}, {1, 3, 4}, {0, 3, 4}, {0, 2, 5}};
static_assert(kNear32Shapes == BIE_NEAR32_SHAPES, "shape count of the public header");
constexpr int kNear32CompChunk = 2048;  // splits with more sources use compensated tile accumulation
constexpr int kDiscSplits = 8;        // source splits per wall point of the wall-discrepancy kernel
constexpr int kCorrLanes = 8;         // lanes per target in k_correct (a power of two <= 32)
constexpr int kVelSplits = 8;         // source splits per body in the velocity extraction
constexpr int kDotChunk = 256;        // vector entries per partial dot product (chunks never span cells)
constexpr int kMaxProxy = 256;
constexpr int kMaxColl = 128;
constexpr int kCloseSlots = 8;        // close body images per target node
constexpr int kMaxRho = 4096;         // largest fine-rule factor of the close evaluation (a power of two)
constexpr int kCloseAccNodes = 4096;  // source nodes per CTA of k_close_blocks (shared accumulators)
constexpr int kMaxBodyNodes = 16384;  // nodes per body
constexpr int kPcMaxNodes = 1024;     // nodes of the contact-block preconditioner: [A_SS | I] (67 MB) stays in L2
constexpr int kMaxCells = 4096;
constexpr int kWallStride = 24;       // doubles per wall point of the wall table (see k_wall_table)
constexpr int kNetHidden = 64;        // hidden width of the warm-start network
constexpr int kNetMaxIn = 16;         // its maximum number of inputs per node
constexpr int kNetFeatures = 13;      // node features of the warm start (features_device)
constexpr int kMaxAug = 3;            // augmentation directions of the first GMRES cycle

// One unit cell of the batch (device table; the host keeps a mirror).
struct Cell {
    double e1[2], e2[2], C[2];
    double mu, gamma, l1, l2;
    double sx[9], sy[9];      // image shifts m e1 + n e2, index (n + 1) * 3 + (m + 1); index 4 is zero
    float sxf[9], syf[9];
    float sxl[9], syl[9];     // sx - sxf, sy - syf: the shifts as double-float pairs
    double inv[4];            // inverse of [e1 e2]: lattice coordinates (s, t) = inv (x - C), row-major
    int node_off, n_nodes, body_off, n_bodies;
    long long part_off[3];    // near-sum partial base (elements) per precision: 0 f32, 1 f64, 2 df64
    int splits[3];            // source splits per precision
    int active;               // solver mask: inactive cells skip the near sums
};

// Close-evaluation storage (Sec. 6.3): per-target slots, compacted pairs,
// 3 N_b doubles (A, B, D of each symmetric 2 x 2 node block) per pair.
struct Close {
    int4* slots = nullptr;        // N x kCloseSlots  (body, image, rho, 0)
    int* count = nullptr;         // N
    int* pair_base = nullptr;     // N + 1
    int4* pairs = nullptr;        // cap_pairs (target, body, image, rho)
    long long* blk_off = nullptr; // cap_pairs
    double* blocks = nullptr;     // cap_doubles
    float* blocks32 = nullptr;    // cap_doubles: the blocks divided by the source weights, single precision
    double* dtab = nullptr;       // Dirichlet tables per distinct node count, rho = 2 .. dtab_rho
    long long* dtab_off = nullptr;  // nb: table base of each body
    int dtab_rho = 0;             // largest rho the tables hold (grown when a pair needs more)
    int* flags = nullptr;         // [total pairs, capacity exceeded, slot overflow, under-resolved,
                                  //  smallest gap below min_gap (8 bytes), largest rho, doubled-cell
                                  //  violations (bit 0: a node beyond the doubled cell, bit 1: a close
                                  //  pair's body image not wholly among its nodes' images), block doubles (8 bytes)]
    int cap_pairs = 0;
    long long cap_doubles = 0;
    bool grow = true;             // storage grows on demand (no close_capacity given)
    int npairs = 0;
    int rho_max = 0;              // largest fine-rule factor of the current pairs
    int under_resolved = 0;       // pairs closer than the finest rule (rho = kMaxRho) resolves
    double min_gap = 0;           // smallest node-to-curve gap below opts.min_gap (else infinity)
    float* dmin = nullptr;        // N: distance to the nearest other curve within the zone (else huge)
    float* dmin_prev = nullptr;   // N: the same for the previous geometry
    float2* ddir = nullptr;       // N: unit vector towards that nearest point (0 if none)
    bool have_dprev = false;
    size_t shm_limit = 0;
    int rule = 0;                 // opts.close_rule: 0 fine trapezoidal rule, 1 barycentric
    double2* bkd = nullptr;       // N: Plemelj diagonal of each body node (barycentric rule)
    double* bcot = nullptr;       // N: spectral-derivative table of each body (barycentric rule)
    double2* bary = nullptr;      // 2 per stored block node: the rule's intermediate vectors
    long long cap_bary = 0;       // bary capacity (double2)
};

// Double-precision source record: position and premultiplied density q = sigma w.
struct __align__(16) Src64 {
    double x, y, z, w;
};

struct Workspace {
    double* sigma = nullptr;    // 2N  staging for host inputs
    double* out = nullptr;      // 2N  staging for host outputs
    Src64* src64 = nullptr;     // N   per node (absolute position)
    float4* src32 = nullptr;    // N, or 4N image records (n_images 4)
    float4* src32n = nullptr;   // N   per node, cell-centred (n_images 4: the wall discrepancy's sources)
    Src64* src64u = nullptr;    // 4N  image records (n_images 4)
    void* srcdf = nullptr;      // N, or 4N image records: double-float source records (32 B)
    double* bodyF = nullptr;    // 3 nb  (F_x, F_y, tau) per body
    void* part = nullptr;       // near-sum partials (see Cell::part_off)
    size_t part_bytes = 0;
    double* gpart = nullptr;    // ncell x kDiscSplits x 8m discrepancy partials
    double* gt = nullptr;       // ncell x 8m  g~ = g0 - g
    unsigned int* dticket = nullptr;  // ncell x 2m last-block counters of k_disc (zero between launches)
    double* xi = nullptr;       // ncell x 2M proxy strengths
    float* xif = nullptr;       // ncell x 2M the same in single precision
    double* T = nullptr;        // 2N traction before the pressure fix
    double* vpart = nullptr;    // nb x kVelSplits x 3 velocity partials
};

// Proxy least-squares fits (Sec. 6.1) of every cell for given lattices:
// stacked matrices, Householder scalars and diagonals, solution operators,
// wall tables (each array holds ncell consecutive blocks).
struct ProxyFit {
    double* A = nullptr;
    double* beta = nullptr;
    double* P = nullptr;
    double* wall = nullptr;
    double* e2 = nullptr;   // 2 x ncell: the lattice vectors e2 the fits are for
    double* yp = nullptr;   // ncell x M x 2 proxy points (on U~'s walls they move with the lattice)
    float2* ypf = nullptr;  // ncell x M proxy points minus the cell centre (single precision)
};

// Per-node image code (n_images 4): bit 0 m0 + 1, bit 1 n0 + 1 (the node's
// four images are (m0 + dm) e1 + (n0 + dn) e2, dm, dn in {0, 1}); bits 2..5
// the index (n + 1) * 3 + (m + 1) of the lattice translate m e1 + n e2 that
// takes the node into U (its wrap).
__host__ __device__ inline int img_m0(int code) { return (code & 1) - 1; }
__host__ __device__ inline int img_n0(int code) { return ((code >> 1) & 1) - 1; }
__host__ __device__ inline int img_wrap(int code) { return (code >> 2) & 15; }
// shift-table index (n + 1) * 3 + (m + 1) of image k = dm + 2 dn of a node
__host__ __device__ inline int img_shift(int code, int k) {
    return (img_n0(code) + (k >> 1) + 1) * 3 + (img_m0(code) + (k & 1) + 1);
}

struct Solver {
    int kmax = 0;
    double* V = nullptr;     // (kmax + 1 + 2 kMaxAug) x 2N: [C~ | Krylov basis | U~]
    double* w = nullptr;     // 2N
    double* r = nullptr;     // 2N
    double* x = nullptr;     // 2N current solution
    double* b = nullptr;     // 2N right-hand side
    double* d = nullptr;     // 2N correction (mixed)
    double* h = nullptr;     // 2 slots of (2 (kmax + 1 + kMaxAug) + 1) x ncell projections, then
                             // (kmax + kMaxAug) x ncell combination coefficients
    double* pinned = nullptr;  // host (page-locked): 2 slots, as on the device
    double* fac = nullptr;   // (4 + 3 kMaxAug) x ncell: normalisation factors, per-cell norms, scratch
    cudaEvent_t ev[2] = {nullptr, nullptr};  // slot k % 2 copied to the host
    unsigned int* ticket = nullptr;  // last-block counter of k_dots (zero between launches)
    double* dpart = nullptr; // (kmax + 2) x nchunks partial dot products
    int4* chunks = nullptr;  // nchunks: (cell, first entry, end entry, 0)
    int2* cell_chunks = nullptr;  // ncell: (first chunk, chunk count)
    int nchunks = 0;
    double* sigma_prev = nullptr;  // 2N the last step's density (warm start of the next)
    double* sigma_prev2 = nullptr; // 2N the density of the step before
    bool have_prev = false, have_prev2 = false;
    double dt_prev = 0;            // the last time step (scales the change features)
    double* aug = nullptr;         // kMaxAug x 2N augmentation directions of the next step
    double* d2 = nullptr;          // 2N the last second-sweep correction (warm_start 2)
    bool have_d2 = false;
    float* feat = nullptr;         // N x kNetFeatures node features
    float* pred = nullptr;         // N x 2 network output
    std::vector<bie_solve_info> cell_info;  // last solve, per cell
};

// Near-sum work list of one precision: one CTA per item (cell, tile, split).
struct NearItems {
    int4* items = nullptr;
    int count = 0;
};

}  // namespace bie

struct bie_ctx {
    int device = 0;
    int sms = 0;                 // streaming multiprocessors of the device (queried at init)
    bool utilde = false;         // opts.n_images == 4: the doubled-cell periodizer
    int srcmul = 1;              // source records per node in the near sums (1, or 4)
    cudaStream_t stream = nullptr;
    bie_opts opts{};
    double t = 0;
    int ncell = 0, nb = 0, N = 0, M = 0, m = 0;
    std::vector<int> n_nodes, offsets;     // per body
    std::vector<double> body_host;         // nb x 8 (a, b, xc, yc, theta, n, off, h)
    std::vector<double> bshape_host;       // nb x 4 (shape, p0, p1, p2)
    std::vector<bie::Cell> cells_h;        // host mirror of the cell table
    std::vector<double> e2_0;              // 2 x ncell lattice vectors e2 at t = 0
    bie::Cell* cells = nullptr;            // device cell table
    bie::Cell* cells_pinned = nullptr;     // page-locked staging copy for uploads
    cudaEvent_t cells_ev = nullptr;        // the last upload has read the staging copy
    int* node_cell = nullptr;              // N
    int* body_cell = nullptr;              // nb
    // device geometry
    double *x = nullptr, *y = nullptr, *nx = nullptr, *ny = nullptr, *w = nullptr, *kap = nullptr;
    int* owner = nullptr;
    double* body = nullptr;
    float4* tgt32 = nullptr;    // N: target x - C, y - C (the translate inside U with n_images 4), normal
    float4* posdf = nullptr;    // N: x - C, y - C as double-float (xh, xl, yh, yl)
    double* xw = nullptr;       // N: target positions of the periodic sums (x, or its translate inside U)
    double* yw = nullptr;
    int* imc = nullptr;         // N: image code (img_m0, img_n0, img_wrap), n_images 4
    int4* bimg = nullptr;       // nb: (min m0, max m0, min n0, max n0) over the body's nodes, n_images 4
    double* bshape = nullptr;   // nb x 4: (shape, p0, p1, p2) -- 0 ellipse (a, b), 1 star (r0, eps, k)
    double* glc = nullptr;      // contour mu_eff: Gauss-Legendre nodes and weights on (-1/2, 1/2) (on demand)
    double* contour_part = nullptr;  // its per-split wall sums (on demand)
    size_t contour_part_n = 0;
    // proxy fits of the current lattices, and of the next time step's (built on
    // a side stream during the current solve)
    double* gl_s = nullptr;     // m Gauss-Legendre nodes on (-1/2, 1/2)
    double* A = nullptr;        // ncell x stacked [Q; lam I], column-major
    double* beta = nullptr;     // ncell x 4M Householder scalars and diagonal
    double* P = nullptr;        // ncell x 2M x 8m solution operators, row-major
    double* wall = nullptr;     // ncell x 2m x 16 wall tables
    double* e2d = nullptr;      // 2 x ncell current lattice vectors e2 (device)
    bie::ProxyFit next;
    cudaStream_t side = nullptr;
    cudaEvent_t next_done = nullptr;
    // the wall discrepancy and proxy strengths of an application run on this
    // stream while the near sum runs on the context's stream (direct launches)
    cudaStream_t aux = nullptr;
    cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
    double* yp = nullptr;       // ncell x M x 2 proxy points of the current fit
    float2* ypf = nullptr;      // ncell x M proxy points minus the cell centre (single precision)
    double* scal = nullptr;     // 3 nb + ncell + 8: velocities, rotation rates, mu_eff
    bie::Workspace ws;
    const double* ws_x = nullptr;  // density whose FP64-class sources, moments and xi the workspace holds
    bie::Solver sv;
    bie::Close cl;
    bie::NearItems near[3];     // 0 single precision, 1 double, 2 double-float
    int shape32 = 0;            // tile shape of the single-precision near sum (kNear32ShapeList)
    int* near_ctr = nullptr;    // work-queue counter of the persistent near sum (batches)
    unsigned long long epoch = 0;  // bumped whenever a kernel argument of the operator application changes
    // contact-block right preconditioner (opts.precond, precond.cu)
    struct {
        int s = 0;                  // nodes in S (0: off for this geometry)
        int cap = 0;                // nodes the block storage holds
        int* nodes = nullptr;       // s: node of each block row pair
        int* pos = nullptr;         // N: block index of each node, -1 outside S
        double* aug = nullptr;      // 2s x 4s: [A_SS | I], after elimination [I | A_SS^-1]
        double* f = nullptr;        // 2s: Gauss-Jordan column
        double* prow = nullptr;     // 4s: Gauss-Jordan pivot row
        int* status = nullptr;      // 1: zero pivot
        double* z = nullptr;        // 2N: preconditioned vector
        double* t = nullptr;        // 2N: combination before preconditioning
    } pc;
    // single-precision application captured as CUDA graphs (opts.graph)
    struct {
        cudaStream_t capture = nullptr;   // stream the capture is recorded on
        cudaGraphExec_t exec[3] = {};     // the three parts of the application
        unsigned long long epoch = ~0ULL; // epoch the graph was captured at
        double* in = nullptr;             // 2N: density the graph reads
        double* out = nullptr;            // 2N: result it writes
        long long kernels = 0;            // launches one replay stands for
    } graph;
    float tune_ms[bie::kNear32Shapes] = {};  // autotuner: median launch time per shape (0 = not timed)
    const bie_net* net = nullptr;  // warm-start network (not owned)
    // target partition across processes (bie_set_partition)
    struct {
        bool on = false;
        int b0 = 0, b1 = 0;          // owned bodies [b0, b1)
        int n0 = 0, n1 = 0;          // their nodes [n0, n1)
        int (*exchange)(double*, int64_t, void*) = nullptr;
        void* user = nullptr;
    } shard;
    // profiling (bie_profile): launch counter and event pairs around near sums
    bool prof = false;
    long long launches = 0;
    std::vector<cudaEvent_t> ev_pool;   // 2 per recorded launch
    std::vector<int> ev_kind;           // 0 = near32, 1 = near64, 2 = near df64 per pair
    int ev_used = 0;
    bie_profile_info prof_acc{};
    std::string err;
    std::vector<double> gl_host;
};

namespace bie {

// status helpers -------------------------------------------------------------
int fail(bie_ctx* c, int code, const std::string& msg);
int cuda_check(bie_ctx* c, cudaError_t e, const char* what);
#define BIE_CUDA(c, call)                                  \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return bie::cuda_check(c, _e, #call); \
    } while (0)
#define BIE_LAUNCH(c, what)                                \
    do {                                                   \
        cudaError_t _e = cudaGetLastError();               \
        if (_e != cudaSuccess) return bie::cuda_check(c, _e, what); \
        ++(c)->launches;                                   \
    } while (0)

// profiling: event pair around a launch (no-op unless bie_profile is on)
int prof_begin(bie_ctx* c, int kind);
int prof_end(bie_ctx* c);
int prof_fold(bie_ctx* c);

// cell table on host and device --------------------------------------------
void cell_set_lattice(Cell& cell, const double* e1, const double* e2);
int upload_cells(bie_ctx* c, cudaStream_t st);

// geometry.cu ---------------------------------------------------------------
int build_geometry(bie_ctx* c);   // nodes from body state
int build_proxy_fit(bie_ctx* c);  // Q, QR of [Q; lam I], P for the current lattices
int build_proxy_fit_to(bie_ctx* c, ProxyFit& f, cudaStream_t st);  // for the lattices f.e2 (device)
int build_wall_table(bie_ctx* c, const double* e2, double* wall, cudaStream_t st);  // e2: device, 2 x ncell
void gauss_legendre_half(int m, std::vector<double>& s);

// close.cu ------------------------------------------------------------------
int build_close(bie_ctx* c);                               // per geometry
int build_dirichlet_tables(bie_ctx* c, int rho_max);       // tables for rho = 2 .. rho_max
int autotune_near32(bie_ctx* c);                           // opts.autotune: time the tile shapes, keep the fastest
int build_precond(bie_ctx* c);                             // opts.precond: contact block of the current geometry
int precond_apply(bie_ctx* c, const double* v, double* z); // z = M^-1 v
void free_precond(bie_ctx* c);
void free_graph(bie_ctx* c);
// T += C sigma; with src32 (the single-precision path's packed sources) the
// own-body and close pairs of the single-precision near sum are also redone
// with positions differenced in double precision
int close_apply(bie_ctx* c, const double* sigma, double* T);
// the single-precision application's assembly: traction, close evaluation,
// pressure fix and rigid completion in two launches (close.cu)
int assemble32(bie_ctx* c, const double* sigma, const Workspace& ws, double* yout);

// apply.cu ------------------------------------------------------------------
// near-sum work items (and partial offsets) for the current cell sizes
int build_near_items(bie_ctx* c);
size_t near_part_bytes(const bie_ctx* c);     // partial buffer the items need
size_t near_part32_elems(const bie_ctx* c);   // single-precision partials of the current items
// y = A sigma for device sigma, y (2N each); precision BIE_FP64 / BIE_MIXED / BIE_DF64
int apply_device(bie_ctx* c, const double* sigma, double* y, int precision);
// single-precision-pair application with caller-provided per-call buffers
int apply_device_ws(bie_ctx* c, const double* sigma, double* y, Workspace& ws);
int rhs_device(bie_ctx* c, double* b);
// double-precision per-node sources, body moments and proxy strengths of sigma
int fp64_moments_and_xi(bie_ctx* c, const double* sigma, bool reuse_ws = false);
// per cell mu_eff by the contour-deformation formula (doubled-cell periodizer; contour.cu)
int mu_eff_contour_device(bie_ctx* c, const double* sigma, double* mu_eff);
// per body v (2 nb), omega (nb); per cell mu_eff (ncell)
int velocities_device(bie_ctx* c, const double* sigma, double* v, double* omega, double* mu_eff,
                      bool reuse_ws = false);

// net.cu --------------------------------------------------------------------
int net_forward_async(bie_ctx* c, const bie_net* n, const float* X, int N, float* Y);
int net_inputs(const bie_net* n);
// N x kNetFeatures node features of the current geometry and stored densities
int features_device(bie_ctx* c, float* X);

// solve.cu ------------------------------------------------------------------
// U: nu augmentation directions (2N each) for the first GMRES cycle when
// starting from zero (use_guess false); may be null.  recycle_second: the
// second refinement sweep (mixed precision) is augmented with the previous
// solve's second-sweep correction, and this one's is kept
int solve_device(bie_ctx* c, const double* b, double* x, bool use_guess, bie_solve_info* info,
                 const double* U = nullptr, int nu = 0, bool recycle_second = false);
int build_dot_chunks(bie_ctx* c);

// small device math shared by the kernels --------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum, 6 operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float z = s - a;
    e = (a - (s - z)) + (b - z);
}

// Double-float numbers (an unevaluated sum hi + lo of two floats).
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

// Packed pairs of floats (PTX .f32x2 on sm_100-family GPUs): one instruction
// performs the same round-to-nearest operation on both halves, so results are
// bit-identical to the scalar operations, with half the issue slots.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The single-precision pair coefficient of the near sum (Eq. Gt without its
// -1/pi): c = (r.n / r^2) (r.q / r^2) for r = (dx, dy), target normal n and
// source strength q; the pair's term is c r.  The 1e-30 floor makes the
// zero-distance self pair contribute 0.  k_near32 and the mixed-precision
// close pass both evaluate pairs through this function, so that the second
// can recompute the first's terms bit for bit.
//
// The y-parts (dy^2 + floor, dy ny, dy qy) are formed first so that a kernel
// can share them between images with the same dy (the three images of a
// lattice row when e1 = (L1, 0)) and still reproduce every term bit for bit.
__device__ __forceinline__ float pair32(float dx, float dy, float nx, float ny, float qx, float qy) {
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, 1e-30f));
    const float rn = fmaf(dx, nx, dy * ny);
    const float rq = fmaf(dx, qx, dy * qy);
    const float inv = rcp_approx(r2);
    return (rn * inv) * (rq * inv);
}

// Star-shaped body (bie_body shape 1): in its own frame the boundary is
// p(t) = r(t) (cos t, sin t), r(t) = r0 (1 + eps cos kt) (Sec. 8 Examples 4-5);
// p, p' and p'' at parameter t.  shp = (1, r0, eps, k).
__device__ inline void star_curve(const double* shp, double t, double& px, double& py, double& dpx, double& dpy,
                                  double& ddpx, double& ddpy) {
    const double r0 = shp[1], eps = shp[2], k = shp[3];
    double st, ct, sk, ck;
    sincos(t, &st, &ct);
    sincos(k * t, &sk, &ck);
    const double r = r0 * (1.0 + eps * ck), dr = -r0 * eps * k * sk, ddr = -r0 * eps * k * k * ck;
    px = r * ct;
    py = r * st;
    dpx = dr * ct - r * st;
    dpy = dr * st + r * ct;
    ddpx = ddr * ct - 2.0 * dr * st - r * ct;
    ddpy = ddr * st + 2.0 * dr * ct - r * st;
}

__host__ __device__ inline void wall_normals(const double* e1, const double* e2, double* nl, double* nd) {
    double l2 = sqrt(e2[0] * e2[0] + e2[1] * e2[1]);
    nl[0] = e2[1] / l2;
    nl[1] = -e2[0] / l2;
    if (nl[0] * e1[0] + nl[1] * e1[1] > 0) { nl[0] = -nl[0]; nl[1] = -nl[1]; }
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1]);
    nd[0] = e1[1] / l1;
    nd[1] = -e1[0] / l1;
    if (nd[0] * e2[0] + nd[1] * e2[1] > 0) { nd[0] = -nd[0]; nd[1] = -nd[1]; }
}

}  // namespace bie
