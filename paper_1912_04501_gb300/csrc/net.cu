// The warm-start network: a per-node multilayer perceptron that maps local
// features of a node (geometry, gap to the nearest other curve, previous
// densities) to a density direction (trained on the change over one time
// step).  It is trained by the kernels below on densities the solver itself
// produced, and
// the solver uses its output only as an extra direction of the first GMRES
// search space (solve.cu), so a poor prediction costs iterations at most.
//
// Architecture (n_in <= kNetMaxIn inputs, H = kNetHidden):
//   a1 = tanh(W1 x + b1)      W1: H x n_in
//   a2 = tanh(W2 a1 + b2)     W2: H x H
//   y  = W3 a2 + b3           W3: 2 x H
// Parameters are one flat array in that order (W row-major).  The kernels
// read the weights in bfloat16 (the training copy keeps FP32 master weights
// and Adam moments).  Layers 1 and 2 and the weight gradients are tcgen05
// tensor-core products (bfloat16 operands, FP32 accumulation in tensor
// memory); tanh, the last layer and the biases are FP32 on the CUDA cores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "bie_internal.cuh"
#include "tc.cuh"

namespace bie {

constexpr int H = kNetHidden;

__host__ __device__ constexpr int net_params(int n_in) { return H * n_in + H + H * H + H + 2 * H + 2; }

struct NetLayout {
    int w1, b1, w2, b2, w3, b3, total;
};

__host__ __device__ inline NetLayout net_layout(int n_in) {
    NetLayout L;
    L.w1 = 0;
    L.b1 = L.w1 + H * n_in;
    L.w2 = L.b1 + H;
    L.b2 = L.w2 + H * H;
    L.w3 = L.b2 + H;
    L.b3 = L.w3 + 2 * H;
    L.total = L.b3 + 2;
    return L;
}

// ---------------------------------------------------------------------------
// Tensor-core kernels (tcgen05).  A tile is 128 nodes, one per thread and one
// per TMEM lane (4 warps = the 4 lane quarters), the M of every MMA.  The
// matrix products take bfloat16 operands and accumulate in float32 in TMEM:
//   layer 1   Z1 [128 x 64] = bf(X) [128 x 16] . W1^T          (1 MMA, K = 16)
//   layer 2   Z2 [128 x 64] = bf(a1) [128 x 64] . W2^T         (4 MMAs)
//   layer 3   y = W3 a2 + b3 per thread (2 outputs: CUDA cores)
// and for the gradient (d3 = 2 w (y - t) per node, unnormalised):
//   d1 GEMM   Z [128 x 64] = bf(d2) [128 x 64] . W2              (4 MMAs)
//   weights   G [128 x 96] += [bf(d2)^T; bf(d1)^T] [128 x 128 nodes] . [bf(a1)^T; bf(x)^T; 1]^T
//             (8 MMAs, K = the tile's 128 nodes): rows 0-63 give gW2 (columns
//             0-63) and gb2 (column 80), rows 64-127 give gW1 (columns 64-79)
//             and gb1 (column 80)
//             G3 [128 x 16] += [bf(a2)^T; 0] . [bf(d3_0); bf(d3_1); 0]^T   (8 MMAs): gW3
// accumulated in TMEM over the CTA's tiles.  bf = round to nearest bfloat16.
// ---------------------------------------------------------------------------
constexpr int kTcTile = 128;     // nodes per tile
constexpr int kTcThreads = 128;  // one thread per node of the tile
constexpr int kK1 = 16;          // layer-1 K: the inputs padded to 16

static_assert(H == 64 && kNetMaxIn <= kK1, "the tensor-core tiles assume 64 hidden units and <= 16 inputs");

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ void st_bf16(uint8_t* p, float v) { *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_row16(uint8_t* base, int r, int k0, int kext, const uint32_t* pk) {
    *reinterpret_cast<uint4*>(base + tc::kmajor_off(r, k0, kext)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

// shared memory (bytes) common to both kernels
constexpr uint32_t kSmXA = 0;                          // 128 x 16 bf(x)      A of layer 1
constexpr uint32_t kSmW1 = kSmXA + kTcTile * kK1 * 2;  // 64 x 16 W1          B of layer 1
constexpr uint32_t kSmA1 = kSmW1 + H * kK1 * 2;        // 128 x 64 bf(a1)     A of layer 2
constexpr uint32_t kSmW2 = kSmA1 + kTcTile * H * 2;    // 64 x 64 W2 [k][j]   B of layer 2
constexpr uint32_t kSmFwdEnd = kSmW2 + H * H * 2;
// the gradient kernel's operands after those
constexpr uint32_t kSmW2T = kSmFwdEnd;                 // 64 x 64 W2^T [j][k] B of the d1 GEMM
constexpr uint32_t kSmD2 = kSmW2T + H * H * 2;         // 128 x 64 bf(d2)     A of the d1 GEMM
constexpr uint32_t kSmAS = kSmD2 + kTcTile * H * 2;    // 128 x 128           A of the weight GEMM
constexpr uint32_t kSmBS = kSmAS + 128 * kTcTile * 2;  // 96 x 128            B of the weight GEMM
constexpr uint32_t kSmA3 = kSmBS + 96 * kTcTile * 2;   // 128 x 128 (64 used) A of the W3 GEMM
constexpr uint32_t kSmB3 = kSmA3 + 128 * kTcTile * 2;  // 16 x 128 (2 used)   B of the W3 GEMM
constexpr uint32_t kSmGradEnd = kSmB3 + 16 * kTcTile * 2;
// parameters in float32, TMEM base, mbarrier, error flag, warp partial sums
constexpr uint32_t kSmParBytes = (2 * H + 2 * H + 2) * 4;
constexpr uint32_t kSmMisc = 64 + 4 * 4 * 4;

__host__ __device__ constexpr uint32_t par_off(uint32_t end) { return (end + 15) & ~15u; }
// forward: 3 CTAs per SM at most (3 x 128 TMEM columns), however small the footprint
constexpr uint32_t kFwdSmem = 60 * 1024;
constexpr uint32_t kGradSmem = par_off(kSmGradEnd) + kSmParBytes + kSmMisc;
static_assert(par_off(kSmFwdEnd) + kSmParBytes + kSmMisc <= kFwdSmem, "forward shared memory");
static_assert(kGradSmem <= 227 * 1024, "gradient shared memory");

struct TcShared {
    float *b1, *b2, *w3, *b3, *part;
    uint32_t* tslot;
    uint64_t* mbar;
    int* err;
};

__device__ inline TcShared tc_shared(uint8_t* sm, uint32_t end) {
    TcShared s;
    s.b1 = reinterpret_cast<float*>(sm + par_off(end));
    s.b2 = s.b1 + H;
    s.w3 = s.b2 + H;
    s.b3 = s.w3 + 2 * H;
    uint8_t* misc = sm + par_off(end) + kSmParBytes;
    s.tslot = reinterpret_cast<uint32_t*>(misc);
    s.mbar = reinterpret_cast<uint64_t*>(misc + 8);
    s.err = reinterpret_cast<int*>(misc + 16);
    s.part = reinterpret_cast<float*>(misc + 64);  // 4 warps x 4
    return s;
}

// weights into the operand tiles (bf16) and parameters (f32); W2T only for the gradient
__device__ inline void tc_load_weights(const __nv_bfloat16* __restrict__ wb, int n_in, uint8_t* sm, const TcShared& S,
                                       bool w2t) {
    const NetLayout L = net_layout(n_in);
    const int t = threadIdx.x;
    for (int e = t; e < H * kK1; e += kTcThreads) {
        const int j = e / kK1, f = e % kK1;
        *reinterpret_cast<__nv_bfloat16*>(sm + kSmW1 + tc::kmajor_off(j, f, kK1)) =
            f < n_in ? wb[L.w1 + j * n_in + f] : __float2bfloat16_rn(0.f);
    }
    for (int e = t; e < H * H; e += kTcThreads) {
        const int k = e / H, j = e % H;
        *reinterpret_cast<__nv_bfloat16*>(sm + kSmW2 + tc::kmajor_off(k, j, H)) = wb[L.w2 + e];
        if (w2t) *reinterpret_cast<__nv_bfloat16*>(sm + kSmW2T + tc::kmajor_off(j, k, H)) = wb[L.w2 + e];
    }
    for (int e = t; e < H; e += kTcThreads) {
        S.b1[e] = __bfloat162float(wb[L.b1 + e]);
        S.b2[e] = __bfloat162float(wb[L.b2 + e]);
        S.w3[e] = __bfloat162float(wb[L.w3 + e]);
        S.w3[H + e] = __bfloat162float(wb[L.w3 + H + e]);
    }
    if (t < 2) S.b3[t] = __bfloat162float(wb[L.b3 + t]);
}

// the CTA's set-up: mbarrier, error flag, TMEM columns (warp 0); returns the TMEM base
__device__ inline uint32_t tc_setup(const TcShared& S, uint32_t ncols) {
    if (threadIdx.x == 0) {
        tc::mbar_init(S.mbar, 1);
        *S.err = 0;
    }
    if (threadIdx.x < 32) tc::tmem_alloc(S.tslot, ncols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *S.tslot;
}

// operands written -> the MMAs issued by thread 0 -> completion waited for by
// every thread (bounded); false (and the CTA's error flag set) on timeout
template <class Issue>
__device__ inline bool tc_step(const TcShared& S, uint32_t& phase, Issue issue) {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        issue();
        tc::commit(S.mbar);
    }
    if (!tc::mbar_wait(S.mbar, phase)) *S.err = 1;
    phase ^= 1;
    tc::fence_after_sync();
    __syncthreads();
    return *S.err == 0;
}

// release TMEM; a CTA whose wait timed out first waits (bounded) for its MMAs
__device__ inline void tc_teardown(const TcShared& S, uint32_t tmem, uint32_t ncols, uint32_t phase, int* err) {
    tc::fence_before_sync();
    __syncthreads();
    if (*S.err) tc::mbar_wait(S.mbar, phase ^ 1, 1 << 20);
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, ncols);
    if (threadIdx.x == 0 && *S.err) atomicExch(err, 1);
}

// layer 1 operand: node i's inputs in bfloat16, zero padded (and, for the
// gradient, their transpose into rows 64.. of the weight GEMM's B)
__device__ inline void tc_inputs(const float* __restrict__ X, int n_in, int i, int N, uint8_t* sm, bool grad) {
    const int t = threadIdx.x;
    float x[kK1];
#pragma unroll
    for (int f = 0; f < kK1; ++f) x[f] = (i < N && f < n_in) ? X[(size_t)i * n_in + f] : 0.f;
    uint32_t pk[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) pk[q] = pack_bf16(x[2 * q], x[2 * q + 1]);
    st_row16(sm + kSmXA, t, 0, kK1, pk);
    st_row16(sm + kSmXA, t, 8, kK1, pk + 4);
    if (grad)
#pragma unroll
        for (int f = 0; f < kK1; ++f) st_bf16(sm + kSmBS + tc::kmajor_off(H + f, t, kTcTile), x[f]);
}

__device__ inline uint64_t desc_k(uint32_t addr, int kext) { return tc::sdesc(addr, 128, (uint32_t)kext * 16); }

// layer 1 and 2 MMAs issued by thread 0
__device__ inline void issue_layer1(uint32_t sbase, uint32_t d1) {
    tc::mma_bf16(d1, desc_k(sbase + kSmXA, kK1), desc_k(sbase + kSmW1, kK1), tc::idesc_bf16(128, H), 0);
}
__device__ inline void issue_layer2(uint32_t sbase, uint32_t d2) {
#pragma unroll
    for (int s = 0; s < H / 16; ++s)
        tc::mma_bf16(d2, desc_k(sbase + kSmA1 + 256 * s, H), desc_k(sbase + kSmW2 + 256 * s, H),
                     tc::idesc_bf16(128, H), s > 0);
}

// layer-1 epilogue: a1 = tanh(z1 + b1) in bfloat16 into row t of layer 2's A
// (and, for the gradient, its transpose into rows 0..63 of the weight GEMM's B)
__device__ inline void tc_layer1_out(uint32_t taddr, const TcShared& S, uint8_t* sm, bool grad) {
    const int t = threadIdx.x;
#pragma unroll
    for (int c = 0; c < H / 16; ++c) {
        float z[16];
        tc::tmem_ld16(taddr + 16 * c, z);
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            pk[q] = pack_bf16(tanhf(z[2 * q] + S.b1[16 * c + 2 * q]), tanhf(z[2 * q + 1] + S.b1[16 * c + 2 * q + 1]));
        st_row16(sm + kSmA1, t, 16 * c, H, pk);
        st_row16(sm + kSmA1, t, 16 * c + 8, H, pk + 4);
        if (grad)
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t w = pk[q >> 1];
                const uint16_t h = (q & 1) ? (uint16_t)(w >> 16) : (uint16_t)(w & 0xFFFFu);
                *reinterpret_cast<uint16_t*>(sm + kSmBS + tc::kmajor_off(16 * c + q, t, kTcTile)) = h;
            }
    }
}

// Inference: y (N x 2) = net(x (N x n_in)) with the bfloat16 roundings of
// the header comment; persistent over tiles.
__global__ void __launch_bounds__(kTcThreads, 1)
k_net_forward(const __nv_bfloat16* __restrict__ wb, int n_in, const float* __restrict__ X, int N,
              float* __restrict__ Y, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const TcShared S = tc_shared(sm, kSmFwdEnd);
    tc_load_weights(wb, n_in, sm, S, false);
    const uint32_t tmem = tc_setup(S, 128);
    const int t = threadIdx.x, warp = t >> 5;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sbase = tc::smem_u32(sm);
    uint32_t phase = 0;
    const int ntiles = (N + kTcTile - 1) / kTcTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * kTcTile + t;
        tc_inputs(X, n_in, i, N, sm, false);
        if (!tc_step(S, phase, [&] { issue_layer1(sbase, tmem); })) break;
        tc_layer1_out(tmem + lane, S, sm, false);
        if (!tc_step(S, phase, [&] { issue_layer2(sbase, tmem + H); })) break;
        float y0 = S.b3[0], y1 = S.b3[1];
#pragma unroll
        for (int c = 0; c < H / 16; ++c) {
            float z[16];
            tc::tmem_ld16(tmem + H + lane + 16 * c, z);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = 16 * c + q;
                const float a2 = tanhf(z[q] + S.b2[k]);
                y0 = fmaf(S.w3[k], a2, y0);
                y1 = fmaf(S.w3[H + k], a2, y1);
            }
        }
        if (i < N) {
            Y[2 * (size_t)i] = y0;
            Y[2 * (size_t)i + 1] = y1;
        }
    }
    tc_teardown(S, tmem, 128, phase, err);
}

// Training: loss L = sum_i w_i |y_i - t_i|^2 / sum_i w_i over the batch and
// its gradient, with the bfloat16 roundings of the header comment.  Each CTA
// takes tiles blockIdx.x, blockIdx.x + gridDim.x, ..., accumulates its
// weight gradients in TMEM and writes them, with its partial loss, bias-3
// gradient and weight sum, to part[block]; k_net_reduce adds the blocks in
// order and normalises.
__global__ void __launch_bounds__(kTcThreads, 1)
k_net_grad(const __nv_bfloat16* __restrict__ wb, int n_in, const float* __restrict__ X, const float* __restrict__ T,
           const float* __restrict__ Wt, int N, float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const NetLayout L = net_layout(n_in);
    const TcShared S = tc_shared(sm, kSmGradEnd);
    tc_load_weights(wb, n_in, sm, S, true);
    const int t = threadIdx.x, warp = t >> 5;
    // fixed parts of the weight GEMMs' operands: B's ones row (80) and zero
    // rows (81..95), the zero upper half of A3 and rows 2..15 of B3
    for (int e = t; e < 16 * kTcTile; e += kTcThreads) {
        const int r = e / kTcTile, n = e % kTcTile;
        st_bf16(sm + kSmBS + tc::kmajor_off(80 + r, n, kTcTile), r == 0 ? 1.f : 0.f);
        if (r >= 2) st_bf16(sm + kSmB3 + tc::kmajor_off(r, n, kTcTile), 0.f);
    }
    for (int e = t; e < 64 * kTcTile; e += kTcThreads)
        st_bf16(sm + kSmA3 + tc::kmajor_off(64 + e / kTcTile, e % kTcTile, kTcTile), 0.f);
    const uint32_t tmem = tc_setup(S, 256);
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sbase = tc::smem_u32(sm);
    const uint32_t dZ = tmem, dZ2 = tmem + H, dG = tmem + 128, dG3 = tmem + 224;
    uint32_t phase = 0;
    float acc_l = 0.f, acc_w = 0.f, acc_g0 = 0.f, acc_g1 = 0.f;  // this node slot's loss, weight, gb3
    const int ntiles = (N + kTcTile - 1) / kTcTile;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int i = tile * kTcTile + t;
        const bool valid = i < N;
        tc_inputs(X, n_in, i, N, sm, true);
        if (!tc_step(S, phase, [&] { issue_layer1(sbase, dZ); })) break;
        tc_layer1_out(dZ + lane, S, sm, true);
        if (!tc_step(S, phase, [&] { issue_layer2(sbase, dZ2); })) break;
        // y, then d3 = 2 w (y - t) (zero for rows past N)
        float y0 = S.b3[0], y1 = S.b3[1];
#pragma unroll
        for (int c = 0; c < H / 16; ++c) {
            float z[16];
            tc::tmem_ld16(dZ2 + lane + 16 * c, z);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = 16 * c + q;
                const float a2 = tanhf(z[q] + S.b2[k]);
                y0 = fmaf(S.w3[k], a2, y0);
                y1 = fmaf(S.w3[H + k], a2, y1);
            }
        }
        float d0 = 0.f, d1 = 0.f;
        if (valid) {
            const float w = Wt[i];
            const float e0 = y0 - T[2 * (size_t)i], e1 = y1 - T[2 * (size_t)i + 1];
            acc_l += w * (e0 * e0 + e1 * e1);
            acc_w += w;
            d0 = 2.f * w * e0;
            d1 = 2.f * w * e1;
            acc_g0 += d0;
            acc_g1 += d1;
        }
        st_bf16(sm + kSmB3 + tc::kmajor_off(0, t, kTcTile), d0);
        st_bf16(sm + kSmB3 + tc::kmajor_off(1, t, kTcTile), d1);
        // d2 = (d3 W3) (1 - a2^2): bf(d2) as row t of the d1 GEMM's A and column t
        // of rows 0..63 of the weight GEMM's A; bf(a2) as column t of A3
#pragma unroll
        for (int c = 0; c < H / 16; ++c) {
            float z[16];
            tc::tmem_ld16(dZ2 + lane + 16 * c, z);
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
                float dv[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = 16 * c + q + u;
                    const float a2 = tanhf(z[q + u] + S.b2[k]);
                    st_bf16(sm + kSmA3 + tc::kmajor_off(k, t, kTcTile), a2);
                    dv[u] = (d0 * S.w3[k] + d1 * S.w3[H + k]) * (1.f - a2 * a2);
                    st_bf16(sm + kSmAS + tc::kmajor_off(k, t, kTcTile), dv[u]);
                }
                pk[q >> 1] = pack_bf16(dv[0], dv[1]);
            }
            st_row16(sm + kSmD2, t, 16 * c, H, pk);
            st_row16(sm + kSmD2, t, 16 * c + 8, H, pk + 4);
        }
        // Z = bf(d2) W2, then d1 = Z (1 - a1^2) with the rounded a1 of layer 2's A
        if (!tc_step(S, phase, [&] {
#pragma unroll
                for (int s = 0; s < H / 16; ++s)
                    tc::mma_bf16(dZ, desc_k(sbase + kSmD2 + 256 * s, H), desc_k(sbase + kSmW2T + 256 * s, H),
                                 tc::idesc_bf16(128, H), s > 0);
            }))
            break;
#pragma unroll
        for (int c = 0; c < H / 16; ++c) {
            float z[16];
            tc::tmem_ld16(dZ + lane + 16 * c, z);
            const uint4 lo = *reinterpret_cast<const uint4*>(sm + kSmA1 + tc::kmajor_off(t, 16 * c, H));
            const uint4 hi = *reinterpret_cast<const uint4*>(sm + kSmA1 + tc::kmajor_off(t, 16 * c + 8, H));
            const uint32_t a[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t bits = (q & 1) ? (a[q >> 1] & 0xFFFF0000u) : (a[q >> 1] << 16);
                const float a1 = __uint_as_float(bits);
                st_bf16(sm + kSmAS + tc::kmajor_off(H + 16 * c + q, t, kTcTile), z[q] * (1.f - a1 * a1));
            }
        }
        // weight gradients, accumulated over the tiles in TMEM
        const uint32_t acc = it > 0 ? 1u : 0u;
        if (!tc_step(S, phase, [&] {
#pragma unroll
                for (int s = 0; s < kTcTile / 16; ++s) {
                    tc::mma_bf16(dG, desc_k(sbase + kSmAS + 256 * s, kTcTile), desc_k(sbase + kSmBS + 256 * s, kTcTile),
                                 tc::idesc_bf16(128, 96), acc | (s > 0));
                    tc::mma_bf16(dG3, desc_k(sbase + kSmA3 + 256 * s, kTcTile),
                                 desc_k(sbase + kSmB3 + 256 * s, kTcTile), tc::idesc_bf16(128, 16), acc | (s > 0));
                }
            }))
            break;
    }
    float* P = part + (size_t)blockIdx.x * (L.total + 2);
    if (*S.err == 0 && it > 0) {
        // TMEM -> this CTA's partial gradient
        float v[16];
        if (warp < 2) {  // rows k = 0..63: gW2[k][.], gb2[k], gW3[.][k]
            const int k = t;
#pragma unroll
            for (int c = 0; c < H / 16; ++c) {
                tc::tmem_ld16(dG + lane + 16 * c, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) P[L.w2 + k * H + 16 * c + q] = v[q];
            }
            tc::tmem_ld16(dG + lane + 80, v);
            P[L.b2 + k] = v[0];
            tc::tmem_ld16(dG3 + lane, v);
            P[L.w3 + k] = v[0];
            P[L.w3 + H + k] = v[1];
        } else {  // rows 64 + j: gW1[j][.], gb1[j]
            const int j = t - 64;
            tc::tmem_ld16(dG + lane + 64, v);
            for (int f = 0; f < n_in; ++f) P[L.w1 + j * n_in + f] = v[f];
            tc::tmem_ld16(dG + lane + 80, v);
            P[L.b1 + j] = v[0];
        }
    }
    // loss, weight and gb3 sums: warps, then the warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_l += __shfl_xor_sync(0xffffffffu, acc_l, o);
        acc_w += __shfl_xor_sync(0xffffffffu, acc_w, o);
        acc_g0 += __shfl_xor_sync(0xffffffffu, acc_g0, o);
        acc_g1 += __shfl_xor_sync(0xffffffffu, acc_g1, o);
    }
    if ((t & 31) == 0) {
        S.part[4 * warp] = acc_l;
        S.part[4 * warp + 1] = acc_w;
        S.part[4 * warp + 2] = acc_g0;
        S.part[4 * warp + 3] = acc_g1;
    }
    __syncthreads();
    if (t == 0) {
        float l = 0.f, w = 0.f, g0 = 0.f, g1 = 0.f;
        for (int k = 0; k < kTcThreads / 32; ++k) {
            l += S.part[4 * k];
            w += S.part[4 * k + 1];
            g0 += S.part[4 * k + 2];
            g1 += S.part[4 * k + 3];
        }
        P[L.b3] = g0;
        P[L.b3 + 1] = g1;
        P[L.total] = l;
        P[L.total + 1] = w;
    }
    tc_teardown(S, tmem, 256, phase, err);
}

// g[p] = (sum over blocks of part[block][p], in block order) / (sum of the
// weights), p <= total (the last entry is the loss).  The block partials were
// formed with the raw weights w_i, so this normalises loss and gradient to
// L = sum_i w_i |y_i - t_i|^2 / sum_i w_i.
__global__ void k_net_reduce(const float* __restrict__ part, int nblocks, int total, float* __restrict__ g) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > total) return;
    const int stride = total + 2;
    double s = 0, ws = 0;
    for (int b = 0; b < nblocks; ++b) {
        s += part[(size_t)b * stride + p];
        ws += part[(size_t)b * stride + total + 1];
    }
    g[p] = ws > 0 ? (float)(s / ws) : 0.f;
}

// Adam (Kingma & Ba) on the FP32 master weights, then their bfloat16 copy.
__global__ void k_net_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, float* __restrict__ m1,
                           float* __restrict__ m2, const float* __restrict__ g, int n, float lr, float beta1,
                           float beta2, float eps, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float gp = g[p];
    const float a = beta1 * m1[p] + (1.f - beta1) * gp;
    const float b = beta2 * m2[p] + (1.f - beta2) * gp * gp;
    m1[p] = a;
    m2[p] = b;
    const float wn = w[p] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[p] = wn;
    wb[p] = __float2bfloat16_rn(wn);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) wb[p] = __float2bfloat16_rn(w[p]);
}


}  // namespace bie

using namespace bie;

struct bie_net {
    int device = 0;
    int n_in = 0, n_params = 0;
    cudaStream_t stream = nullptr;
    float* w = nullptr;             // FP32 master weights
    __nv_bfloat16* wb = nullptr;    // bfloat16 weights read by the kernels
    float* m1 = nullptr;
    float* m2 = nullptr;
    float* g = nullptr;             // n_params + 1 (loss)
    float* part = nullptr;          // per-block partial gradients
    int part_blocks = 0;
    int sms = 0;                    // streaming multiprocessors of the device
    int* tc_err = nullptr;          // set by a kernel whose tensor-core wait timed out
    long long adam_t = 0;
    std::string err;
};

namespace {

int net_fail(bie_net* n, int code, const std::string& m) {
    if (n) n->err = m;
    return code;
}

#define NET_CUDA(n, call)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess)                                                              \
            return net_fail(n, _e == cudaErrorMemoryAllocation ? BIE_ENOMEM : BIE_ECUDA,    \
                            std::string(#call) + ": " + cudaGetErrorString(_e));            \
    } while (0)

void net_free(bie_net* n) {
    void* ptrs[] = {n->w, n->wb, n->m1, n->m2, n->g, n->part, n->tc_err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// the forward's grid: at most 3 CTAs per SM (3 x 128 TMEM columns), each
// over every gridDim-th tile
int forward_grid(const bie_net* n, int N) {
    return std::min((N + kTcTile - 1) / kTcTile, 3 * std::max(1, n->sms));
}

// waits for the network's stream; an error if a tensor-core wait timed out
int check_tc(bie_net* n) {
    int flag = 0;
    NET_CUDA(n, cudaMemcpyAsync(&flag, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    if (flag) return net_fail(n, BIE_ECUDA, "tensor-core completion wait timed out");
    return BIE_OK;
}

int ensure_part(bie_net* n, int blocks) {
    if (blocks <= n->part_blocks) return BIE_OK;
    if (n->part) cudaFree(n->part);
    n->part = nullptr;
    n->part_blocks = 0;
    NET_CUDA(n, cudaMalloc((void**)&n->part, (size_t)blocks * (n->n_params + 2) * sizeof(float)));
    n->part_blocks = blocks;
    return BIE_OK;
}

}  // namespace

extern "C" {

int bie_net_init(bie_net** out, int32_t n_in, int32_t device) {
    if (!out) return BIE_EINVAL;
    *out = nullptr;
    if (n_in < 1 || n_in > kNetMaxIn) return BIE_EINVAL;
    bie_net* n = new (std::nothrow) bie_net();
    if (!n) return BIE_ENOMEM;
    n->device = device;
    n->n_in = n_in;
    n->n_params = net_params(n_in);
    int rc = BIE_OK;
    auto al = [&](void** p, size_t bytes) {
        if (rc) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? BIE_ENOMEM : BIE_ECUDA;
        else cudaMemset(*p, 0, bytes);
    };
    if (cudaSetDevice(device) != cudaSuccess) rc = BIE_ECUDA;
    al((void**)&n->w, n->n_params * sizeof(float));
    al((void**)&n->wb, n->n_params * sizeof(__nv_bfloat16));
    al((void**)&n->m1, n->n_params * sizeof(float));
    al((void**)&n->m2, n->n_params * sizeof(float));
    al((void**)&n->g, (n->n_params + 1) * sizeof(float));
    al((void**)&n->tc_err, sizeof(int));
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = BIE_ECUDA;
    if (!rc && cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) rc = BIE_ECUDA;
    if (!rc && (cudaFuncSetAttribute(k_net_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(k_net_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) !=
                    cudaSuccess))
        rc = BIE_ECUDA;
    if (rc) {
        net_free(n);
        delete n;
        return rc;
    }
    *out = n;
    return BIE_OK;
}

void bie_net_destroy(bie_net* n) {
    if (!n) return;
    cudaSetDevice(n->device);
    cudaStreamSynchronize(n->stream);
    net_free(n);
    delete n;
}

const char* bie_net_last_error(const bie_net* n) { return n ? n->err.c_str() : "null network"; }

int bie_net_size(const bie_net* n, int32_t* n_in, int32_t* hidden, int32_t* n_params) {
    if (!n) return BIE_EINVAL;
    if (n_in) *n_in = n->n_in;
    if (hidden) *hidden = H;
    if (n_params) *n_params = n->n_params;
    return BIE_OK;
}

int bie_net_set_stream(bie_net* n, void* stream) {
    if (!n) return BIE_EINVAL;
    n->stream = (cudaStream_t)stream;
    return BIE_OK;
}

int bie_net_set_params(bie_net* n, const float* params) {
    if (!n || !params) return BIE_EINVAL;
    NET_CUDA(n, cudaSetDevice(n->device));
    NET_CUDA(n, cudaMemcpyAsync(n->w, params, n->n_params * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    NET_CUDA(n, cudaMemsetAsync(n->m1, 0, n->n_params * sizeof(float), n->stream));
    NET_CUDA(n, cudaMemsetAsync(n->m2, 0, n->n_params * sizeof(float), n->stream));
    k_to_bf16<<<(n->n_params + 255) / 256, 256, 0, n->stream>>>(n->w, n->wb, n->n_params);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    n->adam_t = 0;
    return BIE_OK;
}

int bie_net_get_params(bie_net* n, float* params) {
    if (!n || !params) return BIE_EINVAL;
    NET_CUDA(n, cudaSetDevice(n->device));
    NET_CUDA(n, cudaMemcpyAsync(params, n->w, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return BIE_OK;
}

int bie_net_forward(bie_net* n, const float* X, int32_t N, float* Y) {
    if (!n || (N > 0 && (!X || !Y)) || N < 0) return BIE_EINVAL;
    if (N == 0) return BIE_OK;
    NET_CUDA(n, cudaSetDevice(n->device));
    NET_CUDA(n, cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->stream));
    k_net_forward<<<forward_grid(n, N), kTcThreads, kFwdSmem, n->stream>>>(n->wb, n->n_in, X, N, Y, n->tc_err);
    NET_CUDA(n, cudaGetLastError());
    return check_tc(n);
}

int bie_net_loss_grad(bie_net* n, const float* X, const float* T, const float* W, int32_t N, float* grad,
                      double* loss) {
    if (!n || !X || !T || !W || N <= 0) return BIE_EINVAL;
    NET_CUDA(n, cudaSetDevice(n->device));
    // one CTA per SM at most (its shared memory and 256 TMEM columns), each
    // over every gridDim-th tile
    const int blocks = std::min((N + kTcTile - 1) / kTcTile, std::max(1, n->sms));
    if (int rc = ensure_part(n, blocks)) return rc;
    NET_CUDA(n, cudaMemsetAsync(n->tc_err, 0, sizeof(int), n->stream));
    k_net_grad<<<blocks, kTcThreads, kGradSmem, n->stream>>>(n->wb, n->n_in, X, T, W, N, n->part, n->tc_err);
    NET_CUDA(n, cudaGetLastError());
    k_net_reduce<<<(n->n_params + 256) / 256, 256, 0, n->stream>>>(n->part, blocks, n->n_params, n->g);
    NET_CUDA(n, cudaGetLastError());
    if (grad) NET_CUDA(n, cudaMemcpyAsync(grad, n->g, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    float l = 0;
    NET_CUDA(n, cudaMemcpyAsync(&l, n->g + n->n_params, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    if (int rc = check_tc(n)) return rc;
    if (loss) *loss = l;
    return BIE_OK;
}

int bie_net_adam_step(bie_net* n, double lr, double beta1, double beta2, double eps) {
    if (!n || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return BIE_EINVAL;
    NET_CUDA(n, cudaSetDevice(n->device));
    ++n->adam_t;
    const float c1 = (float)(1.0 - std::pow(beta1, (double)n->adam_t));
    const float c2 = (float)(1.0 - std::pow(beta2, (double)n->adam_t));
    k_net_adam<<<(n->n_params + 255) / 256, 256, 0, n->stream>>>(n->w, n->wb, n->m1, n->m2, n->g, n->n_params,
                                                                 (float)lr, (float)beta1, (float)beta2, (float)eps,
                                                                 c1, c2);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return BIE_OK;
}

}  // extern "C"

namespace bie {

// device-side inference for the solver (no synchronisation)
int net_forward_async(bie_ctx* c, const bie_net* n, const float* X, int N, float* Y) {
    k_net_forward<<<forward_grid(n, N), kTcThreads, kFwdSmem, c->stream>>>(n->wb, n->n_in, X, N, Y, n->tc_err);
    BIE_LAUNCH(c, "k_net_forward");
    return BIE_OK;
}

int net_inputs(const bie_net* n) { return n->n_in; }

// Node features of the warm start (kNetFeatures per node), all dimensionless:
//   0, 1   outward normal n
//   2      curvature x the body's node spacing h_b
//   3, 4   (x - x^c) / max(a, b)
//   5, 6   previous step's density / (mu |gamma|)
//   7, 8   (previous - the one before) / (mu |gamma| dt), dt the last step
//   9      log(d / h_b), d the distance to the nearest other curve within the
//          close zone (else the zone's edge, close_factor h_b)
//   10, 11 unit vector towards that nearest point (0 if none)
//   12     log(d_prev / d) / (|gamma| dt), the closing rate of that gap over
//          the last step (0 if unknown)
__global__ void k_features(int N, const double* __restrict__ nx, const double* __restrict__ ny,
                           const double* __restrict__ kap, const double* __restrict__ x,
                           const double* __restrict__ y, const int* __restrict__ owner,
                           const double* __restrict__ body, const int* __restrict__ node_cell,
                           const Cell* __restrict__ cells, const double2* __restrict__ sp,
                           const double2* __restrict__ sp2, const float* __restrict__ dmin,
                           const float* __restrict__ dmin_prev, const float2* __restrict__ ddir, double zone,
                           double dt, float* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* bd = body + 8 * owner[i];
    const double h = bd[7], R = fmax(bd[0], bd[1]);
    const Cell& cl = cells[node_cell[i]];
    const double g = fmax(fabs(cl.gamma), 1e-300);
    const double sc = 1.0 / (cl.mu * g), sct = sc / dt;
    float f[kNetFeatures];
    f[0] = (float)nx[i];
    f[1] = (float)ny[i];
    f[2] = (float)(kap[i] * h);
    f[3] = (float)((x[i] - bd[2]) / R);
    f[4] = (float)((y[i] - bd[3]) / R);
    const double2 a = sp ? sp[i] : make_double2(0, 0);
    const double2 b = (sp && sp2) ? sp2[i] : a;
    f[5] = (float)(a.x * sc);
    f[6] = (float)(a.y * sc);
    f[7] = (float)((a.x - b.x) * sct);
    f[8] = (float)((a.y - b.y) * sct);
    const double big = zone * h;
    const double d = (dmin[i] < 1e30f) ? fmin((double)dmin[i], big) : big;
    const bool near_ = dmin[i] < 1e30f;
    f[9] = (float)log(fmax(d, 1e-300) / h);
    const float2 dir = near_ ? ddir[i] : make_float2(0.f, 0.f);
    f[10] = dir.x;
    f[11] = dir.y;
    double dp = d;
    if (dmin_prev && dmin_prev[i] < 1e30f) dp = fmin((double)dmin_prev[i], big);
    f[12] = (dmin_prev && near_) ? (float)(log(fmax(dp, 1e-300) / fmax(d, 1e-300)) / (g * dt)) : 0.f;
#pragma unroll
    for (int k = 0; k < kNetFeatures; ++k) X[(size_t)i * kNetFeatures + k] = f[k];
}

int features_device(bie_ctx* c, float* X) {
    const bool p1 = c->sv.have_prev, p2 = c->sv.have_prev && c->sv.have_prev2;
    k_features<<<(c->N + 255) / 256, 256, 0, c->stream>>>(
        c->N, c->nx, c->ny, c->kap, c->x, c->y, c->owner, c->body, c->node_cell, c->cells,
        p1 ? reinterpret_cast<const double2*>(c->sv.sigma_prev) : nullptr,
        p2 ? reinterpret_cast<const double2*>(c->sv.sigma_prev2) : nullptr, c->cl.dmin,
        c->cl.have_dprev ? c->cl.dmin_prev : nullptr, c->cl.ddir, c->opts.close_factor > 0 ? c->opts.close_factor : 10.0,
        c->sv.dt_prev > 0 ? c->sv.dt_prev : 1.0, X);
    BIE_LAUNCH(c, "k_features");
    return BIE_OK;
}

}  // namespace bie
