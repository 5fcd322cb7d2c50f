// Allocation-free entry point: denoise + affine normals for callers that
// cannot call cudaMalloc.  The paper has no counterpart; this is a
// deployment convenience.
//
// Some callers cannot allocate device memory: a plugin inside a host
// application that owns all device memory through its own pool, or a
// real-time loop that must not call cudaMalloc (it can synchronise the device
// and take unbounded time).  sn_create allocates its workspace, so those
// callers use sn_normals_noalloc instead: the denoised plane that sn_run_frame
// keeps in context workspace lives here in a file-scope device array, and
// nothing is allocated by this entry point or by anything it calls.
#include <mutex>

#include "sn_internal.h"

// Largest frame the static scratch holds: rows padded to 4 floats, times H.
#define SN_NOALLOC_MAX_ELEMS (2048 * 1024)

// Denoised disparity scratch, one per device that loads the library; held
// until the process exits.  Every call overwrites the elements it reads
// before reading them, so nothing needs clearing between calls.
static __device__ __align__(256) float g_noalloc_den[SN_NOALLOC_MAX_ELEMS];
// Error word handed to the kernels (they only set bits on failed bounded
// waits); sn_noalloc_check_device reads and clears it.
static __device__ __align__(256) int g_noalloc_err[4];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceScratch {
    bool ready = false;
    float* den = nullptr;
    int* err = nullptr;
};

DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Host code may not use the array's name as a device address: the name is a
// host-side stand-in.  Resolve the real addresses once per device, with that
// device current.
cudaError_t scratch_for_device(DeviceScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch& s = g_dev[dev];
    if (!s.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_den);
        if (e != cudaSuccess) return e;
        s.den = static_cast<float*>(p);
        e = cudaGetSymbolAddress(&p, g_noalloc_err);
        if (e != cudaSuccess) return e;
        s.err = static_cast<int*>(p);
        s.ready = true;
    }
    *out = &s;
    return cudaSuccess;
}

bool ok_buf(const void* p, size_t pitch, size_t min_pitch) {
    return p && ((uintptr_t)p & 15u) == 0 && (pitch & 15u) == 0 && pitch >= min_pitch;
}

}  // namespace

extern "C" sn_status sn_normals_noalloc(const sn_camera* cam, const sn_params* p, int W, int H, const void* disp,
                                        size_t disp_pitch, void* normals, size_t normals_pitch, uint8_t* mask,
                                        size_t mask_pitch, sn_stream stream) {
    sn_params defaults;
    if (!p) {
        sn_default_params(&defaults);
        p = &defaults;
    }
    if (W < 1 || H < 1) return SN_EINVAL;
    const size_t den_pitch_elems = ((size_t)W + 3) & ~(size_t)3;
    if (den_pitch_elems * (size_t)H > (size_t)SN_NOALLOC_MAX_ELEMS) return SN_EINVAL;
    sn::Geo g;
    sn::StarTable t;
    sn_status st = sn::prepare_constants(cam, W, H, p, &g, &t);
    if (st != SN_OK) return st;
    const size_t in_elem = p->in_dtype == SN_IN_F32 ? 4 : 2;
    const size_t n_elem = p->normal_fmt == SN_NORMALS_F32X3 ? 4 : 8;
    if (!ok_buf(disp, disp_pitch, (size_t)W * in_elem) || !ok_buf(normals, normals_pitch, (size_t)W * n_elem) ||
        !ok_buf(mask, mask_pitch, (size_t)W))
        return SN_EINVAL;
    DeviceScratch* s = nullptr;
    if (scratch_for_device(&s) != cudaSuccess) return SN_ECUDA;
    g.err = s->err;
    sn::Marks mk;
    cudaError_t e = sn::launch_denoise(g, disp, disp_pitch, s->den, den_pitch_elems * 4, mask, mask_pitch, stream, mk);
    if (e == cudaSuccess)
        e = sn::launch_affine(g, t, disp, disp_pitch, s->den, den_pitch_elems * 4, normals, normals_pitch, mask,
                              mask_pitch, false, stream, mk);
    return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

// The kernels behind sn_normals_noalloc report a bounded wait that gave up
// by setting bits of g_noalloc_err (they never clear it).  This reads and
// clears the word of the current device after `stream` has finished, with
// two synchronous copies between the symbol and a host variable (nothing is
// allocated).
extern "C" sn_status sn_noalloc_check_device(sn_stream stream) {
    DeviceScratch* s = nullptr;
    if (scratch_for_device(&s) != cudaSuccess) return SN_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return SN_ECUDA;
    int err = 0;
    if (cudaMemcpyFromSymbol(&err, g_noalloc_err, sizeof(int)) != cudaSuccess) return SN_ECUDA;
    if (err == 0) return SN_OK;
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_noalloc_err, &zero, sizeof(int)) != cudaSuccess) return SN_ECUDA;
    return SN_ETIMEOUT;
}
