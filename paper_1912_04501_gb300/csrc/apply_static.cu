// bie_apply_static: the single-precision-pair operator application with no
// device allocation.  Every per-call buffer (source records, near-sum
// partials, wall-discrepancy partials, body moments, proxy strengths,
// traction) lives in one file-scope static device array.  Of the context it
// reads the geometry, proxy fit, close tables and work items; it writes only
// its launch counter and, with bie_profile on, the profiler's event state, so
// calls on one context must not overlap (as for every entry point).  See
// include/bie.h for who needs this and the limits.
#include <mutex>

#include "bie_internal.cuh"

// 4 MiB, held by every GPU that loads the library until the process exits.
#define BIE_STATIC_SCRATCH_BYTES (4u << 20)
#define BIE_STATIC_MAX_NODES 8192
#define BIE_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char bie_static_scratch[BIE_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
void* g_static_addr[BIE_STATIC_MAX_DEVICES] = {};  // device address of the array, per device ordinal

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int bie_apply_static(bie_ctx* c, const double* sigma, double* out) {
    using namespace bie;
    if (!c || !sigma || !out) return BIE_EINVAL;
    const size_t N = (size_t)c->N;
    if (c->N > BIE_STATIC_MAX_NODES)
        return fail(c, BIE_EINVAL, "bie_apply_static: the context has " + std::to_string(c->N) +
                                       " nodes; the static scratch serves at most " +
                                       std::to_string(BIE_STATIC_MAX_NODES));
    if (c->device < 0 || c->device >= BIE_STATIC_MAX_DEVICES)
        return fail(c, BIE_EINVAL, "bie_apply_static: device ordinal out of range");
    // layout of the per-call buffers inside the static array (the doubled-cell
    // periodizer has four image records per node, plus per-node records)
    const size_t b_src32 = round256(N * c->srcmul * sizeof(float4));
    const size_t b_src32n = c->utilde ? round256(N * sizeof(float4)) : 0;
    const size_t b_src64 = round256(N * sizeof(Src64));
    const size_t nc = (size_t)c->ncell;
    const size_t b_part = round256(near_part32_elems(c) * sizeof(float2));
    const size_t b_body = round256(3 * (size_t)c->nb * sizeof(double));
    const size_t b_gpart = round256(nc * kDiscSplits * 8 * c->m * sizeof(double));
    const size_t b_xi = round256(nc * 2 * c->M * sizeof(double));
    const size_t b_xif = round256(nc * 2 * c->M * sizeof(float));
    const size_t b_gt = round256(nc * 8 * c->m * sizeof(double));
    const size_t b_tk = round256(nc * 2 * c->m * sizeof(unsigned int));
    const size_t b_T = round256(2 * N * sizeof(double));
    const size_t need = b_src32 + b_src32n + b_src64 + b_part + b_body + b_gpart + b_xi + b_xif + b_gt + b_tk + b_T;
    if (need > BIE_STATIC_SCRATCH_BYTES)
        return fail(c, BIE_EINVAL, "bie_apply_static: this context needs " + std::to_string(need) +
                                       " bytes of scratch; the static array holds " +
                                       std::to_string((size_t)BIE_STATIC_SCRATCH_BYTES));
    BIE_CUDA(c, cudaSetDevice(c->device));
    unsigned char* base = nullptr;
    {
        // Set-up, once per device, with that device current: in host code the
        // array's name is only a host-side stand-in, so the kernels get the
        // device address from cudaGetSymbolAddress.
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[c->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, bie_static_scratch);
            if (e != cudaSuccess) return cuda_check(c, e, "cudaGetSymbolAddress(bie_static_scratch)");
            g_static_addr[c->device] = p;
        }
        base = static_cast<unsigned char*>(g_static_addr[c->device]);
    }
    // Every buffer below is completely written by this call before it is read
    // (the counters are cleared first), so nothing carries over between calls.
    Workspace ws;
    size_t o = 0;
    ws.src32 = reinterpret_cast<float4*>(base + o);
    o += b_src32;
    if (c->utilde) ws.src32n = reinterpret_cast<float4*>(base + o);
    o += b_src32n;
    ws.src64 = reinterpret_cast<Src64*>(base + o);
    o += b_src64;
    ws.part = base + o;
    ws.part_bytes = b_part;
    o += b_part;
    ws.bodyF = reinterpret_cast<double*>(base + o);
    o += b_body;
    ws.gpart = reinterpret_cast<double*>(base + o);
    o += b_gpart;
    ws.xi = reinterpret_cast<double*>(base + o);
    o += b_xi;
    ws.xif = reinterpret_cast<float*>(base + o);
    o += b_xif;
    ws.gt = reinterpret_cast<double*>(base + o);
    o += b_gt;
    ws.dticket = reinterpret_cast<unsigned int*>(base + o);
    o += b_tk;
    ws.T = reinterpret_cast<double*>(base + o);
    // the wall-discrepancy kernel's last-block counters must start at zero
    // (they return to zero when it finishes)
    BIE_CUDA(c, cudaMemsetAsync(ws.dticket, 0, b_tk, c->stream));
    return apply_device_ws(c, sigma, out, ws);
}
