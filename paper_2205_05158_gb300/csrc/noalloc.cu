// Zero-forcing precoder for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: a baseband pipeline
// that reserves all device memory up front and forbids allocation on its real-time
// path, or a process that hands its device memory to a pool owned by someone else.
// fddpd_precode_noalloc serves them: it needs no plan (a plan owns a workspace) and
// allocates nothing.  The Gram / inverse scratch of the three ZF kernels lives in the
// file-scope array below, of fixed size FDDPD_NOALLOC_SCRATCH_BYTES; every GPU that
// loads the library holds it until the process exits.
//
// In host code `noalloc_scratch` names a host-side stand-in, not device memory, so the
// kernels get its device address from cudaGetSymbolAddress.  That look-up is done
// once per device, by the first call on that device (with the device current), and
// cached; that first call should therefore come before any stream capture.
//
// All calls share the one array and it keeps the last call's contents.  The kernels
// overwrite every scratch entry they read, and the status word that must start at zero
// is cleared by each call.  Calls whose kernels overlap on the GPU (different streams,
// or different host threads without ordering) race on the array.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fddpd.h"
#include "kernels.h"

void fddpd_internal_set_error(const char *msg);

namespace {

static __device__ __align__(256) unsigned char noalloc_scratch[FDDPD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr size_t kStatusBytes = 256;   // status word, then the ZF scratch
std::mutex g_setup_mu;
void *g_device_addr[kMaxDevices];      // device address of noalloc_scratch, per device

int fail(int code, const char *msg) {
    fddpd_internal_set_error(msg);
    return code;
}

}  // namespace

extern "C" int fddpd_precode_noalloc(int M, int K, int N_d, int R, double P_T, const fddpd_c32 *H, fddpd_c32 *W,
                                     float *alpha, void *stream) {
    if (M < 1 || M > 512 || K < 1 || K > 32 || K > M || N_d < 1 || R < 1 || !(P_T > 0))
        return fail(FDDPD_ERR_ARG, "fddpd_precode_noalloc: size out of range");
    if (!H || !W || !alpha) return fail(FDDPD_ERR_ARG, "fddpd_precode_noalloc: null pointer");
    if ((reinterpret_cast<uintptr_t>(H) & 7) || (reinterpret_cast<uintptr_t>(W) & 7) ||
        (reinterpret_cast<uintptr_t>(alpha) & 3))
        return fail(FDDPD_ERR_LAYOUT, "fddpd_precode_noalloc: misaligned pointer");
    fdk::Geo g{};
    g.M = M;
    g.K = K;
    g.N_d = N_d;
    g.P_T = P_T;
    const long nbins = (long)R * N_d;
    const size_t need = kStatusBytes + fdk::zf_scratch_bytes(g, nbins);
    if (need > FDDPD_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "fddpd_precode_noalloc: %ld subcarriers x %d users need %zu bytes of scratch, more than the "
                 "%u-byte static array",
                 nbins, K, need, (unsigned)FDDPD_NOALLOC_SCRATCH_BYTES);
        return fail(FDDPD_ERR_UNSUPPORTED, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(FDDPD_ERR_CUDA, "fddpd_precode_noalloc: no usable current device");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_device_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(FDDPD_ERR_CUDA, "fddpd_precode_noalloc: cudaGetSymbolAddress failed");
            }
            g_device_addr[dev] = p;
        }
        base = g_device_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = static_cast<int *>(base);
    void *scratch = static_cast<unsigned char *>(base) + kStatusBytes;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = fdk::zf_build(g, R, reinterpret_cast<const c32 *>(H), reinterpret_cast<c32 *>(W), alpha, status, scratch,
                          nullptr, nullptr, fdk::OUT_F32, st);
    int h_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof msg, "fddpd_precode_noalloc: %s", cudaGetErrorString(e));
        return fail(FDDPD_ERR_CUDA, msg);
    }
    if (h_status) return fail(FDDPD_ERR_SINGULAR, "fddpd_precode_noalloc: a Gram matrix is not positive definite");
    return FDDPD_OK;
}
