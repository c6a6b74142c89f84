// pide2d_jump_static: the jump sum B_w U without any device allocation.
//
// Some callers cannot call cudaMalloc: for example a pricing plugin loaded
// into a host process whose memory manager owns the whole device and
// forbids outside allocations, or a latency-critical service that must not
// allocate after start-up (cudaMalloc can synchronise the device and its
// latency is unbounded).  The regular entry points take a caller-owned
// workspace, which still requires the caller to obtain device memory.  This
// entry point needs none: its scratch is a fixed, file-scope device array of
// 7.2 MB that the library carries on every GPU where it is loaded, until
// the process exits.  That limits it to N <= 256.
//
// It runs the same kernels as pide2d_apply_jump (FP64): the weight spectrum
// is rebuilt from the caller's weights on every call, then one
// zero-padded FFT correlation of the interior of U.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/pide2d.h"
#include "common.cuh"
#include "internal.h"

namespace pide {
void set_global_error(const std::string& msg);
}

using namespace pide;

namespace {

constexpr int kStaticMaxN = 256;
constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr int kP = 2 * kStaticMaxN;
constexpr int kH = kP / 2 + 1;
constexpr int kLd = (kStaticMaxN + 1 + 31) / 32 * 32;
// byte offsets of the scratch regions at the maximum size (smaller grids use a prefix of each)
constexpr size_t kOffS = 0;                                                 // spectrum, column groups x (P+2) rows
constexpr size_t kNg = (size_t)spectrum_groups<double>(kP);
constexpr size_t kGb = cgroup_bytes<double>();
constexpr size_t kOffWt = kOffS + al256(kNg * (kP + 2) * kGb);              // FP64 row spectra of Omega
constexpr size_t kOffWh = kOffWt + al256(kNg * kP * kGb);                   // conj(omega-hat) / P^2
constexpr size_t kOffTw = kOffWh + al256(kNg * kP * kGb);                   // twiddles
constexpr size_t kOffX = kOffTw + al256((size_t)tw_entries(kP) * 16);      // U as FP64 state field
constexpr size_t kOffOut = kOffX + al256((size_t)(kStaticMaxN + 1) * kLd * 8);
constexpr size_t kStaticBytes = kOffOut + al256((size_t)(kStaticMaxN + 1) * kLd * 8);

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

// The scratch.  In host code this name is only a host-side stand-in for
// the device array; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_jump_scratch[kStaticBytes];

namespace {

pide2d_status fail(const std::string& m, pide2d_status s) {
    set_global_error(m);
    return s;
}

// Device address of the scratch on the current device; looked up once per
// device (the first call on a device), then cached.
pide2d_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(std::string("cudaGetDevice: ") + cudaGetErrorString(e), PIDE2D_ERR_CUDA);
    if (dev < 0 || dev >= kMaxDevices) return fail("device index out of range", PIDE2D_ERR_ARG);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_jump_scratch);
        if (e != cudaSuccess || !p)
            return fail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e), PIDE2D_ERR_CUDA);
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PIDE2D_OK;
}

}  // namespace

#define PIDE_STATIC_CUDA(call)                                                         \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(std::string(#call) + ": " + cudaGetErrorString(e_), PIDE2D_ERR_CUDA); \
    } while (0)

extern "C" pide2d_status pide2d_jump_static(int n, const double* omega, const double* U, double* out,
                                            void* cuda_stream) {
    if (n < 8 || n > kStaticMaxN || (n & (n - 1)) != 0)
        return fail("pide2d_jump_static: n must be a power of two in [8, 256] (the static scratch is sized for "
                    "n = 256)", PIDE2D_ERR_ARG);
    if (!omega || !U || !out) return fail("pide2d_jump_static: NULL pointer", PIDE2D_ERR_ARG);
    void* base_v = nullptr;
    const pide2d_status st = scratch_address(&base_v);
    if (st != PIDE2D_OK) return st;
    char* base = static_cast<char*>(base_v);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    Geometry g{};
    g.N = n;
    g.P = 2 * n;
    g.rows = g.P + 2;
    g.ng = spectrum_groups<double>(g.P);
    g.nge = n / rgroup<double>();
    g.ldS = (n + 1 + 31) / 32 * 32;
    g.ldR = g.ldS;
    g.eoff = n / 2 + 3;
    void* S = base + kOffS;
    void* Wt = base + kOffWt;
    void* Wh = base + kOffWh;
    void* tw = base + kOffTw;
    double* X = reinterpret_cast<double*>(base + kOffX);
    double* OUT = reinterpret_cast<double*>(base + kOffOut);

    // conj(fft2(Omega zero-padded)) / P^2 (eq. 3.13); every entry read below
    // is written earlier in this call, so nothing needs clearing
    PIDE_STATIC_CUDA(launch_twiddles<double>(g.P, tw, s));
    Geometry gd = g;
    gd.rows = g.P;
    FwdArgs<double> wa{};
    wa.g = gd;
    wa.mode = FWD_WEIGHTS;
    wa.omega = omega;
    wa.S = Wt;
    wa.pair0 = 0;
    wa.npairs = n / 2;
    wa.tw = tw;
    PIDE_STATIC_CUDA(launch_row_forward<double>(wa, s));
    PIDE_STATIC_CUDA(launch_weights_col<double>(gd, Wt, Wh, nullptr, tw, s));

    // U -> state field, then one zero-padded correlation sweep
    PIDE_STATIC_CUDA(cudaMemcpy2DAsync(OUT, (size_t)g.ldS * 8, U, (size_t)(n + 1) * 8, (size_t)(n + 1) * 8, n + 1,
                                       cudaMemcpyDeviceToDevice, s));
    PIDE_STATIC_CUDA(launch_state_from_double<double>(g, OUT, g.ldS, X, s));
    FwdArgs<double> fa{};
    fa.g = g;
    fa.mode = FWD_FULL0;
    fa.Y = X;
    fa.S = S;
    fa.pair0 = 0;
    fa.npairs = n + 1;
    fa.tw = tw;
    PIDE_STATIC_CUDA(launch_row_forward<double>(fa, s));
    ColArgs<double> ca{};
    ca.g = g;
    ca.mode = COL_FULL;
    ca.S = S;
    ca.Wh = Wh;
    ca.rlo = 0;
    ca.rhi = g.P + 2;
    ca.tw = tw;
    PIDE_STATIC_CUDA(launch_col<double>(ca, s));
    InvArgs<double> ia{};
    ia.g = g;
    ia.mode = INV_OUT;
    ia.do_resid = 0;
    ia.S = S;
    ia.out = OUT;
    ia.tw = tw;
    PIDE_STATIC_CUDA(launch_row_inverse<double>(ia, s));
    PIDE_STATIC_CUDA(cudaMemcpy2DAsync(out + (n + 1) + 1, (size_t)(n + 1) * 8, OUT + g.ldS + 1, (size_t)g.ldS * 8,
                                       (size_t)(n - 1) * 8, n - 1, cudaMemcpyDeviceToDevice, s));
    return PIDE2D_OK;
}
