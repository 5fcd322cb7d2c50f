// C ABI of the surface-normal library: argument checks, context and
// workspace management, and the stage entry points declared in sn.h.
#include <vector>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "sn_gate_internal.h"
#include "sn_internal.h"

namespace {
constexpr int kStages = 4;         // kernel launches of one sn_run_frame
constexpr int kProfFrames = 4096;  // frames recorded between two sn_stage_times calls
constexpr int kAux = 4;            // side streams the component passes of sn_run_frame fork onto
constexpr int kHostSlots = 4;      // device staging sets of sn_run_frame_host

// Device staging of one sn_run_frame_host frame; `done` is recorded after
// its copies back to the host.
struct HostSlot {
    void* in;
    size_t in_p;
    void* nrm;
    size_t nrm_p;
    float* pts;
    size_t pts_p;
    int32_t* lab;
    size_t lab_p;
    uint8_t* mask;
    size_t mask_p;
    int32_t* count;
    cudaEvent_t done;
    bool used;
};
const char* const kStageNames[kStages] = {"frame", "ccl_local", "ccl_merge", "ccl_flatten"};
}  // namespace

struct sn_ctx {
    sn_camera cam;
    int W, H;
    sn_params p;
    int device;
    sn::Geo geo;
    sn::StarTable star;
    sn::Workspace ws;
    unsigned long long launches;
    bool star8;  // the star table is the compile-time M = 8, s = 10 ray set
    sn::GateDev gate;    // learned gate weights (learned contexts)
    float* gate_theta;   // their FP32 source on the device
    void* net_img;       // the weights as the learned kernel's shared memory holds them
    const float* log2tab;  // the library's table of log2 of every code (learned contexts)
    sn::GateView gv;       // what the learned kernels read (set by sn_load_gate_weights)
    int* star_pm;        // prefix moments of the star's rays (device)
    bool gate_loaded;
    bool prof;
    cudaEvent_t* ev;  // kProfFrames x (kStages + 1)
    int prof_frames;
    // The component passes read only the disparity, so sn_run_frame runs
    // them on a side stream forked from the caller's (events fork and join),
    // concurrently with the frame kernel; frames take the side streams in turn.
    cudaStream_t aux[kAux];
    cudaEvent_t fork_ev[kAux], join_ev[kAux];
    int aux_next;
    HostSlot hs[kHostSlots];  // allocated by the first sn_run_frame_host
    bool hs_ready;
    int hs_next;
    char msg[512];
};

namespace {

void free_host_slots(sn_ctx* c) {
    for (int i = 0; i < kHostSlots; i++) {
        HostSlot& h = c->hs[i];
        cudaFree(h.in);
        cudaFree(h.nrm);
        cudaFree(h.pts);
        cudaFree(h.lab);
        cudaFree(h.mask);
        cudaFree(h.count);
        if (h.done) cudaEventDestroy(h.done);
        h = HostSlot{};
    }
    c->hs_ready = false;
}

int kfix(float k) { return (int)nearbyint((double)k * 65536.0); }

sn_status fail(sn_ctx* c, sn_status st, const char* what) {
    if (c) snprintf(c->msg, sizeof(c->msg), "%s", what);
    return st;
}

sn_status cuda_fail(sn_ctx* c, cudaError_t e, const char* where) {
    if (c) snprintf(c->msg, sizeof(c->msg), "%s: %s", where, cudaGetErrorString(e));
    return SN_ECUDA;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

sn_status check_buf(sn_ctx* c, const void* p, size_t pitch, size_t elem, const char* name) {
    if (!p) return fail(c, SN_EINVAL, name);
    if (!aligned16(p) || (pitch & 15u) != 0 || pitch < (size_t)c->W * elem) {
        char buf[160];
        snprintf(buf, sizeof(buf), "%s: pointer must be 16-byte aligned, pitch a multiple of 16 and >= %zu bytes",
                 name, (size_t)c->W * elem);
        return fail(c, SN_EINVAL, buf);
    }
    return SN_OK;
}

size_t in_elem(int dtype) { return dtype == SN_IN_F32 ? 4 : 2; }
size_t nrm_elem(int fmt) { return fmt == SN_NORMALS_F32X3 ? 4 : 8; }

// Star-fill offsets: direction j at angle 2 pi j / M, step k at
// (round(k cos), round(k sin)) with halves away from zero (C round()).
void star_offsets(int M, int s, int8_t* ou, int8_t* ov) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < M; j++) {
        const double th = two_pi * (double)j / (double)M;
        const double c = cos(th), sn_ = sin(th);
        for (int k = 1; k <= s; k++) {
            ou[j * s + k - 1] = (int8_t)round(k * c);
            ov[j * s + k - 1] = (int8_t)round(k * sn_);
        }
    }
}

// Classifies every table entry for the kernels (see sn::StarTable).
bool build_star(int M, int s, sn::StarTable& T) {
    memset(&T, 0, sizeof(T));
    T.n = M * s;
    star_offsets(M, s, T.ou, T.ov);
    for (int e = 0; e < T.n; e++) {
        const int j = e / s, k = e % s;
        if (k > 0 && T.ou[e] == T.ou[e - 1] && T.ov[e] == T.ov[e - 1]) {
            T.cls[e] = 0;
            continue;
        }
        // rays (other than j) that reach the same offset
        bool shared = false;
        for (int f = 0; f < T.n; f++)
            if (f / s != j && T.ou[f] == T.ou[e] && T.ov[f] == T.ov[e]) shared = true;
        if (!shared) {
            T.cls[e] = 1;
            continue;
        }
        int b = -1;
        for (int q = 0; q < T.nshared; q++)
            if (T.sou[q] == T.ou[e] && T.sov[q] == T.ov[e]) b = q;
        if (b < 0) {
            if (T.nshared >= sn::kMaxShared) return false;
            b = T.nshared++;
            T.sou[b] = T.ou[e];
            T.sov[b] = T.ov[e];
        }
        T.cls[e] = 2;
        T.bit[e] = (uint8_t)b;
    }
    return true;
}

}  // namespace

namespace sn {

// With w within 1 ulp (2^-23 relative) of 1/D and thr = fl(K 2^-16 / Dc),
// the computed spread fl(w_hi - w_lo) differs from 1/Dmin - 1/Dmax by at
// most 2^-23 (1/Dmin + 1/Dmax) + 2^-24 (spread + thr).  Near the threshold
// (spread ~ thr = kappa / Dc with kappa = K / 2^16) Dmin >= Dc / (1 + kappa),
// so the error is at most thr 2^-23 (2 (1 + kappa) / kappa + 1).  The band
// is four times that.
void cd_band(int K, float* hi, float* lo) {
    if (K <= 0) {
        *hi = 1.0f;
        *lo = 1.0f;
        return;
    }
    const double kappa = K / 65536.0;
    const double e = 4.0 * ldexp(1.0, -23) * (2.0 * (1.0 + kappa) / kappa + 1.0);
    *hi = (float)(1.0 + e);
    *lo = (float)(1.0 - e);
}

// ST constants: F = 256 fx B as the FP64 product (256 fx) B (the order the
// exact Laplacian test uses), its FP32 copy for the banded fast test, and t.
static void set_st(sn::Geo& g, const sn_camera* cam, float t) {
    g.st_F = (256.0 * cam->fx) * cam->baseline;
    g.st_Ff = (float)g.st_F;
    g.st_t = (double)t;
    g.st_tf = t;
}

// Validates camera, size and parameters like sn_create and fills the kernel
// constants, without touching the device (used by the allocation-free entry
// point; err is left null for the caller to set).
sn_status prepare_constants(const sn_camera* cam, int W, int H, const sn_params* p, Geo* g, StarTable* t) {
    if (!cam || !p || !g || !t || W < 1 || H < 1 || W > 16384 || H > 16384) return SN_EINVAL;
    if (!(cam->fx > 0) || !(cam->fy > 0) || !(cam->baseline > 0) || !isfinite(cam->cx) || !isfinite(cam->cy) ||
        !isfinite(cam->fx) || !isfinite(cam->fy) || !isfinite(cam->baseline))
        return SN_EINVAL;
    if (p->r_denoise < 1 || p->r_denoise > 4 || p->r_affine < 1 || p->r_affine > 15) return SN_EINVAL;
    if (p->support < SN_SUPPORT_FIXED || p->support > SN_SUPPORT_STARFILL_ST) return SN_EINVAL;
    if (!(p->st_t >= 0.0f) || !isfinite(p->st_t)) return SN_EINVAL;
    if (p->dirs < 4 || p->dirs > kMaxDirs || p->steps < 1 || p->steps > kMaxSteps) return SN_EINVAL;
    if (!(p->k_cd >= 0 && p->k_cd <= 1) || !(p->k_pair >= 0 && p->k_pair <= 1) ||
        !(p->k_range >= 0 && p->k_range <= 1) || !(p->tau >= 0 && p->tau <= 1))
        return SN_EINVAL;
    if (p->in_dtype < SN_IN_F32 || p->in_dtype > SN_IN_U16X256) return SN_EINVAL;
    if (p->normal_fmt != SN_NORMALS_F32X3 && p->normal_fmt != SN_NORMALS_SNORM16X4) return SN_EINVAL;
    if (p->learned) return SN_ENOTSUP;
    if (!build_star(p->dirs, p->steps, *t)) return SN_ENOTSUP;
    memset(g, 0, sizeof(*g));
    g->W = W;
    g->w_rcp = w_reciprocal(W);
    g->H = H;
    g->in_dtype = p->in_dtype;
    g->r_d = p->r_denoise;
    g->r_a = p->r_affine;
    g->support = p->support;
    g->dirs = p->dirs;
    g->steps = p->steps;
    g->K_cd = kfix(p->k_cd);
    g->K_pair = kfix(p->k_pair);
    g->K_range = kfix(p->k_range);
    cd_band(g->K_cd, &g->cd_hi, &g->cd_lo);
    g->normal_fmt = p->normal_fmt;
    g->fx = (float)cam->fx;
    g->fy = (float)cam->fy;
    g->cx = (float)cam->cx;
    g->cy = (float)cam->cy;
    g->B = (float)cam->baseline;
    g->fy_over_fx = (float)(cam->fy / cam->fx);
    g->inv_fx = (float)(1.0 / cam->fx);
    g->B_fx_over_fy = (float)(cam->baseline * cam->fx / cam->fy);
    g->fxB = (float)(cam->fx * cam->baseline);
    g->dfx = cam->fx;
    g->dfy = cam->fy;
    g->dcx = cam->cx;
    g->dcy = cam->cy;
    g->dB = cam->baseline;
    set_st(*g, cam, p->st_t);
    g->walk_limit = kWalkLimitDefault;
    return SN_OK;
}

}  // namespace sn

extern "C" {

int sn_version(void) { return (0 << 16) | 3; }

void sn_default_params(sn_params* p) {
    if (!p) return;
    p->r_denoise = 2;
    p->r_affine = 4;
    p->support = SN_SUPPORT_STARFILL_CD;
    p->dirs = 8;
    p->steps = 10;
    p->k_cd = 0.1f;
    p->k_pair = 0.05f;
    p->k_range = 0.05f;
    p->tau = 0.9f;
    p->in_dtype = SN_IN_F32;
    p->normal_fmt = SN_NORMALS_F32X3;
    p->learned = 0;
    p->st_t = 0.1f;
}

const char* sn_status_string(sn_status s) {
    switch (s) {
        case SN_OK: return "ok";
        case SN_EINVAL: return "invalid argument";
        case SN_ENOMEM: return "out of device memory";
        case SN_ECUDA: return "CUDA error";
        case SN_ETIMEOUT: return "bounded device wait gave up";
        case SN_EBUSY: return "busy (admission refused)";
        case SN_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

const char* sn_last_error(const sn_ctx* c) { return c ? c->msg : "null context"; }

sn_status sn_rcp_table(float* out, int n) {
    if (!out || n < sn::kDMax + 1) return SN_EINVAL;
    return sn::rcp_codes(out) == cudaSuccess ? SN_OK : SN_ECUDA;
}

int sn_star_offsets(int dirs, int steps, int8_t* ou, int8_t* ov) {
    if (dirs < 1 || dirs > sn::kMaxDirs || steps < 1 || steps > sn::kMaxSteps || !ou || !ov) return -1;
    star_offsets(dirs, steps, ou, ov);
    return dirs * steps;
}

sn_status sn_create(const sn_camera* cam, int W, int H, const sn_params* pin, sn_ctx** out) {
    if (!out) return SN_EINVAL;
    *out = nullptr;
    if (!cam || W < 1 || H < 1 || W > 16384 || H > 16384) return SN_EINVAL;
    if (!(cam->fx > 0) || !(cam->fy > 0) || !(cam->baseline > 0) || !isfinite(cam->cx) || !isfinite(cam->cy) ||
        !isfinite(cam->fx) || !isfinite(cam->fy) || !isfinite(cam->baseline))
        return SN_EINVAL;
    sn_params p;
    if (pin)
        p = *pin;
    else
        sn_default_params(&p);
    if (p.r_denoise < 1 || p.r_denoise > 4 || p.r_affine < 1 || p.r_affine > 15) return SN_EINVAL;
    if (p.support < SN_SUPPORT_FIXED || p.support > SN_SUPPORT_STARFILL_ST) return SN_EINVAL;
    if (!(p.st_t >= 0.0f) || !isfinite(p.st_t)) return SN_EINVAL;
    if (p.dirs < 4 || p.dirs > sn::kMaxDirs || p.steps < 1 || p.steps > sn::kMaxSteps) return SN_EINVAL;
    if (!(p.k_cd >= 0 && p.k_cd <= 1) || !(p.k_pair >= 0 && p.k_pair <= 1) || !(p.k_range >= 0 && p.k_range <= 1) ||
        !(p.tau >= 0 && p.tau <= 1))
        return SN_EINVAL;
    if (p.in_dtype < SN_IN_F32 || p.in_dtype > SN_IN_U16X256) return SN_EINVAL;
    if (p.normal_fmt != SN_NORMALS_F32X3 && p.normal_fmt != SN_NORMALS_SNORM16X4) return SN_EINVAL;
    if (p.learned != 0 && p.learned != 1) return SN_EINVAL;
    // the gate certifies the full 9x9 window and 5x5 denoise window of the
    // default star-fill configuration
    if (p.learned && (p.support != SN_SUPPORT_STARFILL_CD || p.dirs != 8 || p.steps != 10 || p.r_denoise != 2 ||
                      p.r_affine != 4))
        return SN_ENOTSUP;

    sn_ctx* c = new (std::nothrow) sn_ctx();
    if (!c) return SN_ENOMEM;
    c->cam = *cam;
    c->W = W;
    c->H = H;
    c->p = p;
    cudaGetDevice(&c->device);
    if (!build_star(p.dirs, p.steps, c->star)) {
        delete c;
        return SN_ENOTSUP;
    }
    c->star8 = sn::star_is_m8(c->star, p.dirs, p.steps);
    sn::Geo& g = c->geo;
    g.W = W;
    g.H = H;
    g.in_dtype = p.in_dtype;
    g.r_d = p.r_denoise;
    g.r_a = p.r_affine;
    g.support = p.support;
    g.dirs = p.dirs;
    g.steps = p.steps;
    g.K_cd = kfix(p.k_cd);
    g.K_pair = kfix(p.k_pair);
    g.K_range = kfix(p.k_range);
    sn::cd_band(g.K_cd, &g.cd_hi, &g.cd_lo);
    g.normal_fmt = p.normal_fmt;
    g.fx = (float)cam->fx;
    g.fy = (float)cam->fy;
    g.cx = (float)cam->cx;
    g.cy = (float)cam->cy;
    g.B = (float)cam->baseline;
    g.fy_over_fx = (float)(cam->fy / cam->fx);
    g.inv_fx = (float)(1.0 / cam->fx);
    g.B_fx_over_fy = (float)(cam->baseline * cam->fx / cam->fy);
    g.fxB = (float)(cam->fx * cam->baseline);
    g.dfx = cam->fx;
    g.dfy = cam->fy;
    g.dcx = cam->cx;
    g.dcy = cam->cy;
    g.dB = cam->baseline;
    sn::set_st(g, cam, p.st_t);
    g.walk_limit = sn::kWalkLimitDefault;
    g.w_rcp = sn::w_reciprocal(W);

    cudaError_t e = cudaMalloc(&c->ws.err, 2 * sizeof(int));
    if (e == cudaSuccess) {
        c->ws.count = c->ws.err + 1;
        e = cudaMemset(c->ws.err, 0, 2 * sizeof(int));
    }
    if (e == cudaSuccess) {
        c->ws.den_pitch = ((size_t)W * 4 + 15) & ~(size_t)15;
        e = cudaMalloc(&c->ws.den, c->ws.den_pitch * H);
    }
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (int i = 0; i < kAux && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithPriority(&c->aux[i], cudaStreamNonBlocking, prio_hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork_ev[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) {
        std::vector<int> pm((size_t)p.dirs * (p.steps + 1) * 6);
        sn::star_prefix_moments(c->star, p.dirs, p.steps, pm.data());
        e = cudaMalloc((void**)&c->star_pm, sizeof(int) * pm.size());
        if (e == cudaSuccess) e = cudaMemcpy(c->star_pm, pm.data(), sizeof(int) * pm.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && p.learned) {
        e = sn::gate_alloc(c->gate);
        if (e == cudaSuccess) e = cudaMalloc(&c->gate_theta, sizeof(float) * sn::kGateParams);
        if (e == cudaSuccess) e = cudaMalloc(&c->net_img, sn::kNetImageBytes);
        if (e == cudaSuccess) e = sn::log2_table(&c->log2tab);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        sn_destroy(c);
        return SN_ENOMEM;
    }
    g.err = c->ws.err;
    g.star_pm = c->star_pm;
    snprintf(c->msg, sizeof(c->msg), "ok");
    *out = c;
    return SN_OK;
}

sn_status sn_destroy(sn_ctx* c) {
    if (!c) return SN_OK;
    if (c->ev) {
        for (int i = 0; i < kProfFrames * (kStages + 1); i++) cudaEventDestroy(c->ev[i]);
        delete[] c->ev;
    }
    free_host_slots(c);
    for (int i = 0; i < kAux; i++) {
        if (c->aux[i]) cudaStreamDestroy(c->aux[i]);
        if (c->fork_ev[i]) cudaEventDestroy(c->fork_ev[i]);
        if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
    }
    if (c->ws.err) cudaFree(c->ws.err);
    if (c->ws.den) cudaFree(c->ws.den);
    if (c->gate.W1g) sn::gate_free(c->gate);
    if (c->gate_theta) cudaFree(c->gate_theta);
    if (c->net_img) cudaFree(c->net_img);
    if (c->star_pm) cudaFree(c->star_pm);
    delete c;
    return SN_OK;
}

sn_status sn_denoise(sn_ctx* c, const void* disp, size_t dpitch, float* den, size_t denp, uint8_t* mask,
                     size_t mp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, den, denp, 4, "den")) != SN_OK) return st;
    if ((st = check_buf(c, mask, mp, 1, "mask")) != SN_OK) return st;
    sn::Marks mk;
    cudaError_t e = sn::launch_denoise(c->geo, disp, dpitch, den, denp, mask, mp, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_denoise");
}

sn_status sn_affine_normals(sn_ctx* c, const void* disp, size_t dpitch, const float* den, size_t denp,
                            void* nrm, size_t np, uint8_t* mask, size_t mp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, den, denp, 4, "den")) != SN_OK) return st;
    if ((st = check_buf(c, nrm, np, nrm_elem(c->p.normal_fmt), "normals")) != SN_OK) return st;
    if ((st = check_buf(c, mask, mp, 1, "mask")) != SN_OK) return st;
    sn::Marks mk;
    cudaError_t e = sn::launch_affine(c->geo, c->star, disp, dpitch, den, denp, nrm, np, mask, mp, false, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_affine_normals");
}

sn_status sn_cross_normals(sn_ctx* c, const void* disp, size_t dpitch, void* nrm, size_t np, uint8_t* mask,
                           size_t mp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, nrm, np, nrm_elem(c->p.normal_fmt), "normals")) != SN_OK) return st;
    if ((st = check_buf(c, mask, mp, 1, "mask")) != SN_OK) return st;
    sn::Marks mk;
    cudaError_t e = sn::launch_cross(c->geo, disp, dpitch, nrm, np, mask, mp, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_cross_normals");
}

sn_status sn_pca_normals(sn_ctx* c, const void* disp, size_t dpitch, int r, void* nrm, size_t np, uint8_t* mask,
                         size_t mp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    if (r < 1 || r > 7) return fail(c, SN_EINVAL, "pca radius outside 1..7");
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, nrm, np, nrm_elem(c->p.normal_fmt), "normals")) != SN_OK) return st;
    if ((st = check_buf(c, mask, mp, 1, "mask")) != SN_OK) return st;
    sn::Marks mk;
    cudaError_t e = sn::launch_pca(c->geo, disp, dpitch, r, nrm, np, mask, mp, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_pca_normals");
}

sn_status sn_components(sn_ctx* c, const void* disp, size_t dpitch, int32_t* labels, size_t lp, int32_t* ncomp,
                        sn_stream stream) {
    if (!c) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, labels, lp, 4, "labels")) != SN_OK) return st;
    if (ncomp && ((uintptr_t)ncomp & 3u)) return fail(c, SN_EINVAL, "num_components: misaligned");
    sn::Marks mk;
    cudaError_t e = sn::launch_components(c->geo, disp, dpitch, labels, lp, ncomp, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_components");
}

sn_status sn_pointcloud(sn_ctx* c, const float* den, size_t denp, const uint8_t* mask, size_t mp, float* pts,
                        size_t pp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, den, denp, 4, "den")) != SN_OK) return st;
    if ((st = check_buf(c, mask, mp, 1, "mask")) != SN_OK) return st;
    if ((st = check_buf(c, pts, pp, 4, "points")) != SN_OK) return st;
    sn::Marks mk;
    cudaError_t e = sn::launch_points(c->geo, den, denp, mask, mp, pts, pp, stream, mk);
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_pointcloud");
}

sn_status sn_run_frame(sn_ctx* c, const sn_frame_in* in, sn_frame_out* out, sn_stream stream) {
    if (!c || !in || !out) return SN_EINVAL;
    sn_status st;
    if ((st = check_buf(c, in->disp, in->disp_pitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    float* den = out->den;
    size_t denp = out->den_pitch;
    if (den) {
        if ((st = check_buf(c, den, denp, 4, "den")) != SN_OK) return st;
    } else {
        den = c->ws.den;
        denp = c->ws.den_pitch;
    }
    if ((st = check_buf(c, out->normals, out->normals_pitch, nrm_elem(c->p.normal_fmt), "normals")) != SN_OK) return st;
    if ((st = check_buf(c, out->points, out->points_pitch, 4, "points")) != SN_OK) return st;
    if ((st = check_buf(c, out->labels, out->labels_pitch, 4, "labels")) != SN_OK) return st;
    if ((st = check_buf(c, out->mask, out->mask_pitch, 1, "mask")) != SN_OK) return st;
    if (out->num_components && ((uintptr_t)out->num_components & 3u))
        return fail(c, SN_EINVAL, "num_components: misaligned");
    sn::Marks mk;
    if (c->prof && c->prof_frames < kProfFrames) {
        mk.ev = c->ev + (size_t)c->prof_frames * (kStages + 1);
        cudaEventRecord(mk.ev[0], stream);
        mk.n = 1;
        c->prof_frames++;
    }
    sn::FrameOut fo;
    fo.den = out->den;
    fo.denp = out->den_pitch;
    fo.nrm = out->normals;
    fo.np = out->normals_pitch;
    fo.pts = out->points;
    fo.pp = out->points_pitch;
    fo.labels = out->labels;
    fo.lp = out->labels_pitch;
    fo.mask = out->mask;
    fo.mp = out->mask_pitch;
    fo.count = out->num_components;
    (void)den;
    (void)denp;
    sn::GateView gv{};
    if (c->p.learned) {
        if (!c->gate_loaded) return fail(c, SN_EINVAL, "learned context: gate weights not loaded");
        gv = c->gv;
    }
    const sn::GateView* g = c->p.learned ? &gv : nullptr;
    cudaError_t e;
    if (mk.ev) {
        // profiled frames keep all launches on the caller's stream, so that
        // the events between them time each kernel alone
        e = sn::launch_frame(c->geo, c->star, c->star8, in->disp, in->disp_pitch, fo, g, stream, mk);
        if (e == cudaSuccess)
            e = sn::launch_components(c->geo, in->disp, in->disp_pitch, fo.labels, fo.lp, fo.count, stream, mk);
    } else {
        const int i = c->aux_next;
        c->aux_next = (i + 1) % kAux;
        e = cudaEventRecord(c->fork_ev[i], stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux[i], c->fork_ev[i], 0);
        if (e == cudaSuccess)
            e = sn::launch_components(c->geo, in->disp, in->disp_pitch, fo.labels, fo.lp, fo.count, c->aux[i], mk);
        if (e == cudaSuccess) e = cudaEventRecord(c->join_ev[i], c->aux[i]);
        if (e == cudaSuccess) e = sn::launch_frame(c->geo, c->star, c->star8, in->disp, in->disp_pitch, fo, g, stream, mk);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, c->join_ev[i], 0);
    }
    c->launches += mk.launches;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_run_frame");
}

sn_status sn_gate_q(sn_ctx* c, const void* disp, size_t dpitch, float* q, size_t qp, sn_stream stream) {
    if (!c) return SN_EINVAL;
    if (!c->p.learned) return fail(c, SN_EINVAL, "sn_gate_q: context was not created with learned = 1");
    if (!c->gate_loaded) return fail(c, SN_EINVAL, "sn_gate_q: gate weights not loaded");
    sn_status st;
    if ((st = check_buf(c, disp, dpitch, in_elem(c->p.in_dtype), "disp")) != SN_OK) return st;
    if ((st = check_buf(c, q, qp, 4, "q")) != SN_OK) return st;
    const sn::GateView gv = c->gv;
    const sn::FrameOut none{};
    cudaError_t e = sn::launch_learned(c->geo, disp, dpitch, none, gv, q, qp, stream);
    if (e == cudaSuccess) c->launches++;
    return e == cudaSuccess ? SN_OK : cuda_fail(c, e, "sn_gate_q");
}

namespace {

cudaError_t alloc_host_slots(sn_ctx* c) {
    const size_t W = (size_t)c->W, H = (size_t)c->H;
    const bool f32 = c->p.normal_fmt == SN_NORMALS_F32X3;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kHostSlots && e == cudaSuccess; i++) {
        HostSlot& h = c->hs[i];
        e = cudaMallocPitch(&h.in, &h.in_p, W * in_elem(c->p.in_dtype), H);
        if (e == cudaSuccess) e = cudaMallocPitch(&h.nrm, &h.nrm_p, W * nrm_elem(c->p.normal_fmt), f32 ? 3 * H : H);
        if (e == cudaSuccess) e = cudaMallocPitch((void**)&h.pts, &h.pts_p, W * 4, 3 * H);
        if (e == cudaSuccess) e = cudaMallocPitch((void**)&h.lab, &h.lab_p, W * 4, H);
        if (e == cudaSuccess) e = cudaMallocPitch((void**)&h.mask, &h.mask_p, W, H);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h.count, 16);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming);
    }
    return e;
}

}  // namespace

sn_status sn_run_frame_host(sn_ctx* c, const sn_frame_in* in, sn_frame_out* out, sn_stream stream) {
    if (!c || !in || !out) return SN_EINVAL;
    const size_t W = (size_t)c->W, H = (size_t)c->H;
    const bool f32 = c->p.normal_fmt == SN_NORMALS_F32X3;
    const size_t ie = in_elem(c->p.in_dtype), ne = nrm_elem(c->p.normal_fmt);
    if (out->den) return fail(c, SN_EINVAL, "sn_run_frame_host: den must be NULL");
    if (!in->disp || in->disp_pitch < W * ie) return fail(c, SN_EINVAL, "host disp: NULL or pitch too short");
    if (!out->normals || out->normals_pitch < W * ne) return fail(c, SN_EINVAL, "host normals: NULL or pitch too short");
    if (!out->points || out->points_pitch < W * 4) return fail(c, SN_EINVAL, "host points: NULL or pitch too short");
    if (!out->labels || out->labels_pitch < W * 4) return fail(c, SN_EINVAL, "host labels: NULL or pitch too short");
    if (!out->mask || out->mask_pitch < W) return fail(c, SN_EINVAL, "host mask: NULL or pitch too short");
    if (!c->hs_ready) {
        const cudaError_t e = alloc_host_slots(c);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_host_slots(c);
            return fail(c, SN_ENOMEM, "sn_run_frame_host: staging buffers");
        }
        c->hs_ready = true;
    }
    HostSlot& h = c->hs[c->hs_next];
    c->hs_next = (c->hs_next + 1) % kHostSlots;
    cudaError_t e = h.used ? cudaStreamWaitEvent(stream, h.done, 0) : cudaSuccess;
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(h.in, h.in_p, in->disp, in->disp_pitch, W * ie, H, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sn_run_frame_host: copy in");
    sn_frame_in fi{h.in, h.in_p};
    sn_frame_out fo{};
    fo.normals = h.nrm;
    fo.normals_pitch = h.nrm_p;
    fo.points = h.pts;
    fo.points_pitch = h.pts_p;
    fo.labels = h.lab;
    fo.labels_pitch = h.lab_p;
    fo.mask = h.mask;
    fo.mask_pitch = h.mask_p;
    fo.num_components = out->num_components ? h.count : nullptr;
    const sn_status st = sn_run_frame(c, &fi, &fo, stream);
    if (st != SN_OK) return st;
    e = cudaMemcpy2DAsync(out->normals, out->normals_pitch, h.nrm, h.nrm_p, W * ne, f32 ? 3 * H : H,
                          cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out->points, out->points_pitch, h.pts, h.pts_p, W * 4, 3 * H, cudaMemcpyDeviceToHost,
                              stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out->labels, out->labels_pitch, h.lab, h.lab_p, W * 4, H, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out->mask, out->mask_pitch, h.mask, h.mask_p, W, H, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && out->num_components)
        e = cudaMemcpyAsync(out->num_components, h.count, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaEventRecord(h.done, stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sn_run_frame_host: copy out");
    h.used = true;
    return SN_OK;
}

sn_status sn_set_walk_limit(sn_ctx* c, int steps) {
    if (!c) return SN_EINVAL;
    c->geo.walk_limit = steps > 0 ? steps : sn::kWalkLimitDefault;
    return SN_OK;
}

sn_status sn_load_gate_weights(sn_ctx* c, const void* blob, size_t bytes) {
    if (!c || !blob) return SN_EINVAL;
    if (!c->p.learned) return fail(c, SN_EINVAL, "context was not created with learned = 1");
    const unsigned char* b = static_cast<const unsigned char*>(blob);
    const size_t need = 12 + sizeof(float) * (size_t)sn::kGateParams;
    uint32_t ver = 0, n = 0;
    if (bytes >= 12) {
        memcpy(&ver, b + 4, 4);
        memcpy(&n, b + 8, 4);
    }
    if (bytes < need || memcmp(b, "SNGW", 4) != 0 || ver != 1 || n != (uint32_t)sn::kGateParams)
        return fail(c, SN_EINVAL, "not a version-1 gate weights blob of the expected size");
    cudaError_t e = cudaMemcpy(c->gate_theta, b + 12, sizeof(float) * sn::kGateParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = sn::gate_layout(c->gate_theta, c->gate, nullptr);
    if (e == cudaSuccess) {
        sn::GateView gv{};
        gv.W1g = c->gate.W1g;
        gv.W2g = c->gate.W2g;
        gv.b1 = c->gate.b1;
        gv.b2 = c->gate.b2;
        gv.W3 = c->gate.W3;
        gv.b3 = c->gate.b3;
        gv.tau = c->p.tau;
        gv.net = c->net_img;
        gv.log2tab = c->log2tab;
        float theta[sn::kGateParams];
        memcpy(theta, b + 12, sizeof(theta));
        sn::gate_constants(theta, &gv);
        e = sn::launch_net_image(gv, c->net_img, nullptr);
        if (e == cudaSuccess) c->gv = gv;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "sn_load_gate_weights");
    c->gate_loaded = true;
    return SN_OK;
}

sn_status sn_set_profiling(sn_ctx* c, int on) {
    if (!c) return SN_EINVAL;
    if (on && !c->ev) {
        const int n = kProfFrames * (kStages + 1);
        c->ev = new (std::nothrow) cudaEvent_t[n]();
        if (!c->ev) return fail(c, SN_ENOMEM, "profiling events");
        for (int i = 0; i < n; i++) {
            cudaError_t e = cudaEventCreate(&c->ev[i]);
            if (e != cudaSuccess) return cuda_fail(c, e, "sn_set_profiling");
        }
    }
    c->prof = on != 0;
    c->prof_frames = 0;
    return SN_OK;
}

int sn_stage_count(const sn_ctx* c) { return c ? kStages : 0; }

const char* sn_stage_name(const sn_ctx* c, int i) {
    return (c && i >= 0 && i < kStages) ? kStageNames[i] : nullptr;
}

sn_status sn_stage_times(sn_ctx* c, double* ms, int n, int* frames, double* frame_ms, int cap) {
    if (!c || !ms || n < kStages) return SN_EINVAL;
    for (int i = 0; i < kStages; i++) ms[i] = 0.0;
    const int nf = c->prof_frames;
    for (int f = 0; f < nf; f++) {
        cudaEvent_t* e = c->ev + (size_t)f * (kStages + 1);
        cudaError_t err = cudaEventSynchronize(e[kStages]);
        if (err != cudaSuccess) return cuda_fail(c, err, "sn_stage_times");
        for (int i = 0; i < kStages; i++) {
            float t = 0.0f;
            err = cudaEventElapsedTime(&t, e[i], e[i + 1]);
            if (err != cudaSuccess) return cuda_fail(c, err, "sn_stage_times");
            ms[i] += t;
        }
        if (frame_ms && f < cap) {
            float t = 0.0f;
            err = cudaEventElapsedTime(&t, e[0], e[kStages]);
            if (err != cudaSuccess) return cuda_fail(c, err, "sn_stage_times");
            frame_ms[f] = t;
        }
    }
    if (frames) *frames = nf;
    c->prof_frames = 0;
    return SN_OK;
}

uint64_t sn_launch_count(const sn_ctx* c) { return c ? (uint64_t)c->launches : 0; }

sn_status sn_check_device(sn_ctx* c, sn_stream stream) {
    if (!c) return SN_EINVAL;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "sn_check_device");
    int err = 0;
    e = cudaMemcpy(&err, c->ws.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "sn_check_device");
    if (err) {
        cudaMemset(c->ws.err, 0, sizeof(int));
        snprintf(c->msg, sizeof(c->msg), "device error bits 0x%x", err);
        return SN_ETIMEOUT;
    }
    return SN_OK;
}

}  // extern "C"
