// The warm-start network: a per-node multilayer perceptron that maps local
// features of a node (geometry, gap to the nearest other curve, previous
// densities) to a predicted change of the density over one time step.  It is
// trained by the kernels below on densities the solver itself produced, and
// the solver uses its output only as an extra direction of the first GMRES
// search space (solve.cu), so a poor prediction costs iterations at most.
//
// Architecture (n_in <= kNetMaxIn inputs, H = kNetHidden):
//   a1 = tanh(W1 x + b1)      W1: H x n_in
//   a2 = tanh(W2 a1 + b2)     W2: H x H
//   y  = W3 a2 + b3           W3: 2 x H
// Parameters are one flat array in that order (W row-major).  The forward
// passes read the weights in bfloat16 (the training copy keeps FP32 master
// weights and Adam moments); every product and sum is in FP32.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "bie_internal.cuh"

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

// bfloat16 weights -> FP32 shared-memory copy (all threads of the block)
__device__ inline void load_weights(const __nv_bfloat16* __restrict__ wb, int n, float* __restrict__ s) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) s[k] = __bfloat162float(wb[k]);
    __syncthreads();
}

// Inference: one thread per node; y (N x 2) = net(x (N x n_in)).
__global__ void __launch_bounds__(128)
k_net_forward(const __nv_bfloat16* __restrict__ wb, int n_in, const float* __restrict__ X, int N,
              float* __restrict__ Y) {
    extern __shared__ float sw[];
    const NetLayout L = net_layout(n_in);
    load_weights(wb, L.total, sw);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float x[kNetMaxIn];
#pragma unroll
    for (int f = 0; f < kNetMaxIn; ++f) x[f] = f < n_in ? X[(size_t)i * n_in + f] : 0.f;
    float a1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float z = sw[L.b1 + j];
#pragma unroll
        for (int f = 0; f < kNetMaxIn; ++f)
            if (f < n_in) z = fmaf(sw[L.w1 + j * n_in + f], x[f], z);
        a1[j] = tanhf(z);
    }
    float y0 = sw[L.b3], y1 = sw[L.b3 + 1];
    for (int k = 0; k < H; ++k) {
        float z = sw[L.b2 + k];
#pragma unroll
        for (int j = 0; j < H; ++j) z = fmaf(sw[L.w2 + k * H + j], a1[j], z);
        const float a2 = tanhf(z);
        y0 = fmaf(sw[L.w3 + k], a2, y0);
        y1 = fmaf(sw[L.w3 + H + k], a2, y1);
    }
    Y[2 * (size_t)i] = y0;
    Y[2 * (size_t)i + 1] = y1;
}

// Training: loss L = sum_i w_i |y_i - t_i|^2 / sum_i w_i over the batch, its
// gradient with respect to every parameter.  Block of kNetBlock nodes:
// activations and back-propagated errors live in shared memory, each
// weight-gradient entry is summed over the block's nodes by one thread, and
// the block writes its partial gradient (and partial loss) to
// part[block][...]; k_net_reduce adds the blocks in order.
constexpr int kNetBlock = 128;
constexpr int kRow = H + 1;  // padded row of the per-node activation tables

__global__ void __launch_bounds__(kNetBlock)
k_net_grad(const __nv_bfloat16* __restrict__ wb, int n_in, const float* __restrict__ X,
           const float* __restrict__ T, const float* __restrict__ Wt, int N, float* __restrict__ part) {
    extern __shared__ float sm[];
    const NetLayout L = net_layout(n_in);
    float* sw = sm;                                  // L.total weights
    float* A1 = sw + ((L.total + 3) & ~3);           // kNetBlock x kRow: a1, later delta1
    float* A2 = A1 + kNetBlock * kRow;               // kNetBlock x kRow: a2, later delta2
    float* SX = A2 + kNetBlock * kRow;               // kNetBlock x n_in
    float* D3 = SX + kNetBlock * kNetMaxIn;          // kNetBlock x 2
    float* RL = D3 + 2 * kNetBlock;                  // kNetBlock: per-node loss
    float* RW = RL + kNetBlock;                      // kNetBlock: per-node weight
    load_weights(wb, L.total, sw);
    const int t = threadIdx.x;
    const int i = blockIdx.x * kNetBlock + t;
    const bool valid = i < N;
    // forward, one thread per node
    {
        float x[kNetMaxIn];
#pragma unroll
        for (int f = 0; f < kNetMaxIn; ++f) {
            x[f] = (valid && f < n_in) ? X[(size_t)i * n_in + f] : 0.f;
            SX[t * kNetMaxIn + f] = x[f];
        }
        for (int j = 0; j < H; ++j) {
            float z = sw[L.b1 + j];
#pragma unroll
            for (int f = 0; f < kNetMaxIn; ++f)
                if (f < n_in) z = fmaf(sw[L.w1 + j * n_in + f], x[f], z);
            A1[t * kRow + j] = tanhf(z);
        }
        float y0 = sw[L.b3], y1 = sw[L.b3 + 1];
        for (int k = 0; k < H; ++k) {
            float z = sw[L.b2 + k];
            for (int j = 0; j < H; ++j) z = fmaf(sw[L.w2 + k * H + j], A1[t * kRow + j], z);
            const float a2 = tanhf(z);
            A2[t * kRow + k] = a2;
            y0 = fmaf(sw[L.w3 + k], a2, y0);
            y1 = fmaf(sw[L.w3 + H + k], a2, y1);
        }
        float d0 = 0.f, d1 = 0.f, l = 0.f, w = 0.f;
        if (valid) {
            w = Wt[i];
            const float e0 = y0 - T[2 * (size_t)i], e1 = y1 - T[2 * (size_t)i + 1];
            l = w * (e0 * e0 + e1 * e1);
            d0 = 2.f * w * e0;
            d1 = 2.f * w * e1;
        }
        D3[2 * t] = d0;
        D3[2 * t + 1] = d1;
        RL[t] = l;
        RW[t] = w;
    }
    __syncthreads();
    float* P = part + (size_t)blockIdx.x * (L.total + 2);
    // layer 3: dW3[k][c] = sum_n D3[n][c] a2[n][c]; db3
    for (int e = t; e < 2 * H + 2; e += kNetBlock) {
        float s = 0.f;
        if (e < 2 * H) {
            const int c = e / H, k = e - c * H;
            for (int n = 0; n < kNetBlock; ++n) s = fmaf(D3[2 * n + c], A2[n * kRow + k], s);
            P[L.w3 + e] = s;
        } else {
            const int c = e - 2 * H;
            for (int n = 0; n < kNetBlock; ++n) s += D3[2 * n + c];
            P[L.b3 + c] = s;
        }
    }
    __syncthreads();
    // delta2 = (1 - a2^2) W3^T d3, in place of a2
    for (int k = 0; k < H; ++k) {
        const float a2 = A2[t * kRow + k];
        A2[t * kRow + k] = (1.f - a2 * a2) * (sw[L.w3 + k] * D3[2 * t] + sw[L.w3 + H + k] * D3[2 * t + 1]);
    }
    __syncthreads();
    // layer 2: dW2[k][j] = sum_n delta2[n][k] a1[n][j]; db2
    for (int e = t; e < H * H + H; e += kNetBlock) {
        float s = 0.f;
        if (e < H * H) {
            const int k = e / H, j = e - k * H;
            for (int n = 0; n < kNetBlock; ++n) s = fmaf(A2[n * kRow + k], A1[n * kRow + j], s);
            P[L.w2 + e] = s;
        } else {
            const int k = e - H * H;
            for (int n = 0; n < kNetBlock; ++n) s += A2[n * kRow + k];
            P[L.b2 + k] = s;
        }
    }
    __syncthreads();
    // delta1 = (1 - a1^2) W2^T delta2, in place of a1
    {
        float d1[H];
#pragma unroll
        for (int j = 0; j < H; ++j) d1[j] = 0.f;
        for (int k = 0; k < H; ++k) {
            const float d2 = A2[t * kRow + k];
#pragma unroll
            for (int j = 0; j < H; ++j) d1[j] = fmaf(sw[L.w2 + k * H + j], d2, d1[j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const float a1 = A1[t * kRow + j];
            A1[t * kRow + j] = (1.f - a1 * a1) * d1[j];
        }
    }
    __syncthreads();
    // layer 1: dW1[j][f] = sum_n delta1[n][j] x[n][f]; db1
    for (int e = t; e < H * n_in + H; e += kNetBlock) {
        float s = 0.f;
        if (e < H * n_in) {
            const int j = e / n_in, f = e - j * n_in;
            for (int n = 0; n < kNetBlock; ++n) s = fmaf(A1[n * kRow + j], SX[n * kNetMaxIn + f], s);
            P[L.w1 + e] = s;
        } else {
            const int j = e - H * n_in;
            for (int n = 0; n < kNetBlock; ++n) s += A1[n * kRow + j];
            P[L.b1 + j] = s;
        }
    }
    if (t == 0) {
        float s = 0.f, sw_ = 0.f;
        for (int n = 0; n < kNetBlock; ++n) {
            s += RL[n];
            sw_ += RW[n];
        }
        P[L.total] = s;
        P[L.total + 1] = sw_;
    }
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

size_t net_grad_smem(int n_in) {
    const NetLayout L = net_layout(n_in);
    return sizeof(float) * (((L.total + 3) & ~3) + 2 * kNetBlock * kRow + kNetBlock * kNetMaxIn + 4 * kNetBlock);
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
    void* ptrs[] = {n->w, n->wb, n->m1, n->m2, n->g, n->part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
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
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = BIE_ECUDA;
    if (!rc) {
        const size_t smem = net_grad_smem(n_in);
        if (cudaFuncSetAttribute(k_net_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            rc = BIE_ECUDA;
    }
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
    const size_t smem = n->n_params * sizeof(float);
    k_net_forward<<<(N + 127) / 128, 128, smem, n->stream>>>(n->wb, n->n_in, X, N, Y);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return BIE_OK;
}

int bie_net_loss_grad(bie_net* n, const float* X, const float* T, const float* W, int32_t N, float* grad,
                      double* loss) {
    if (!n || !X || !T || !W || N <= 0) return BIE_EINVAL;
    NET_CUDA(n, cudaSetDevice(n->device));
    const int blocks = (N + kNetBlock - 1) / kNetBlock;
    if (int rc = ensure_part(n, blocks)) return rc;
    const size_t smem = net_grad_smem(n->n_in);
    k_net_grad<<<blocks, kNetBlock, smem, n->stream>>>(n->wb, n->n_in, X, T, W, N, n->part);
    NET_CUDA(n, cudaGetLastError());
    k_net_reduce<<<(n->n_params + 256) / 256, 256, 0, n->stream>>>(n->part, blocks, n->n_params, n->g);
    NET_CUDA(n, cudaGetLastError());
    if (grad) NET_CUDA(n, cudaMemcpyAsync(grad, n->g, n->n_params * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    float l = 0;
    NET_CUDA(n, cudaMemcpyAsync(&l, n->g + n->n_params, sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
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
    const size_t smem = n->n_params * sizeof(float);
    k_net_forward<<<(N + 127) / 128, 128, smem, c->stream>>>(n->wb, n->n_in, X, N, Y);
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
