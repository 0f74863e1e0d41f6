// mot_fields_noalloc: the far-field evaluation of mot_fields without any device
// allocation during the call.
//
// Who needs it: code that may not call cudaMalloc / cudaFree at this point, for
// example a host application whose memory pool owns all device memory after
// start-up, or a latency-critical loop where cudaMalloc / cudaFree would
// synchronise the device. mot_fields stages the directions and the result in
// buffers it allocates on every call; this variant stages them in one fixed
// device array compiled into the library instead.
//
// The array (MOT_NOALLOC_FIELD_DOUBLES doubles, 2 MiB) exists on every GPU that
// loads the library and stays there until the process exits. Its device
// address is looked up once per device, by the first call made with that
// device current; make that first call before any stream capture. The address
// is kept for the life of the process, so a device reset (cudaDeviceReset)
// between calls is not supported. All calls
// share the array and it keeps the last call's contents; the kernel writes
// every output element, so nothing has to be cleared, but calls whose work
// overlaps on the GPU race on it and must be serialised by the caller.
#include <mutex>
#include <string>

#include "mot_internal.h"

#define MOT_API extern "C" __attribute__((visibility("default")))

static __device__ __align__(256) double g_field_scratch[MOT_NOALLOC_FIELD_DOUBLES];

namespace mot {
void launch_far_field(mot_handle* h, int n_dir, const double* dirs, double* E, cudaStream_t s);
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_field_scratch on device `dev` (looked up once per device).
cudaError_t scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}
}  // namespace

MOT_API int mot_fields_noalloc(mot_handle* h, const mot_wave* waves, int n_dir, const double* dirs, double* E_out) {
    (void)waves;
    if (!h || !E_out || n_dir < 1 || !dirs) return MOT_EINVAL;
    if (!h->d_dft || h->nfreq == 0) return mot::fail(h, MOT_ESTATE, "no Fourier sums: call mot_set_frequencies and step");
    const size_t ndirs = (size_t)3 * n_dir;
    const size_t nout = (size_t)h->B * h->nfreq * n_dir * 6;
    if (ndirs + nout > (size_t)MOT_NOALLOC_FIELD_DOUBLES)
        return mot::fail(h, MOT_EINVAL,
                         "mot_fields_noalloc: 3*n_dir + 6*B*n_freq*n_dir = " + std::to_string(ndirs + nout) +
                             " doubles exceeds the fixed scratch of " + std::to_string(MOT_NOALLOC_FIELD_DOUBLES) +
                             "; use mot_fields or fewer directions");
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "cudaSetDevice");
    double* base = nullptr;
    e = scratch_address(h->dev, &base);
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "cudaGetSymbolAddress(g_field_scratch)");
    double* d_E = base;             // the result first: it starts on the array's 256-byte boundary
    double* d_dirs = base + nout;   // the directions right after it
    e = cudaMemcpy(d_dirs, dirs, sizeof(double) * ndirs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "cudaMemcpy(directions)");
    // the Fourier sums of the last step, on whatever stream it ran
    e = cudaStreamWaitEvent(0, h->ev_state, 0);
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "cudaStreamWaitEvent");
    mot::launch_far_field(h, n_dir, d_dirs, d_E, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "far-field kernel launch");
    e = cudaMemcpy(E_out, d_E, sizeof(double) * nout, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mot::cuda_fail(h, e, "cudaMemcpy(result)");
    return MOT_OK;
}
