// Serving runtime (include/sn_serve.h): per-camera request queues, slots
// admitted by a device-memory budget, one CUDA graph per slot, several
// streams, a scheduler thread that admits, launches and polls, and a camera
// simulator with Poisson arrivals.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sn_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

size_t pad16(size_t b) { return (b + 15) & ~(size_t)15; }

struct Slot {
    int cam = 0;
    void* d_in = nullptr;
    size_t in_pitch = 0;
    void* d_nrm = nullptr;
    size_t nrm_pitch = 0;
    float* d_pts = nullptr;
    size_t pts_pitch = 0;
    int32_t* d_lab = nullptr;
    size_t lab_pitch = 0;
    uint8_t* d_mask = nullptr;
    size_t mask_pitch = 0;
    int32_t* d_count = nullptr;
    void* h_out = nullptr;  // pinned: normals | points | labels | mask | count
    void* h_nrm = nullptr;
    float* h_pts = nullptr;
    int32_t* h_lab = nullptr;
    uint8_t* h_mask = nullptr;
    int32_t* h_count = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;  // launched, not yet complete
    bool held = false;  // complete, result not yet released by the client
    bool sim = false;
    uint64_t tag = 0;
    double t_arrival = 0.0;
};

struct Req {
    int cam;
    const void* host;
    size_t pitch;
    uint64_t tag;
    double t_arrival;
    bool sim;
};

struct Cam {
    sn_server_camera cfg;
    sn_ctx* ctx = nullptr;
    std::vector<int> slots;
    std::deque<Req> queue;
    size_t in_elem = 4, nrm_bytes_px = 12;
};

}  // namespace

struct sn_server {
    sn_server_config cfg{};
    int device = 0;
    std::vector<Cam> cams;
    std::vector<Slot> slots;
    std::vector<cudaStream_t> streams;
    unsigned rr = 0;
    std::thread thread;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    long long waiting = 0;
    long long inflight = 0;
    std::deque<sn_serve_result> completed;
    std::vector<double> sim_lat;
    long long sim_done_px = 0;
    double sim_last_done = 0.0;
    sn_status err = SN_OK;
};

namespace {

// Slot sizes of a camera's frame (device bytes).
size_t slot_bytes(const Cam& c) {
    const size_t W = c.cfg.W, H = c.cfg.H;
    return H * pad16(W * c.in_elem) + (c.nrm_bytes_px == 12 ? 3 * H * pad16(W * 4) : H * pad16(W * 8)) +
           3 * H * pad16(W * 4) + H * pad16(W * 4) + H * pad16(W) + 256;
}

cudaError_t make_slot(sn_server* s, Cam& c, Slot& sl, cudaStream_t cap) {
    const int W = c.cfg.W, H = c.cfg.H;
    cudaError_t e;
    sl.in_pitch = pad16((size_t)W * c.in_elem);
    sl.nrm_pitch = c.nrm_bytes_px == 12 ? pad16((size_t)W * 4) : pad16((size_t)W * 8);
    const size_t nrm_rows = c.nrm_bytes_px == 12 ? 3 * (size_t)H : (size_t)H;
    sl.pts_pitch = pad16((size_t)W * 4);
    sl.lab_pitch = pad16((size_t)W * 4);
    sl.mask_pitch = pad16((size_t)W);
    if ((e = cudaMalloc(&sl.d_in, sl.in_pitch * H)) != cudaSuccess) return e;
    if ((e = cudaMemset(sl.d_in, 0, sl.in_pitch * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sl.d_nrm, sl.nrm_pitch * nrm_rows)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&sl.d_pts, sl.pts_pitch * 3 * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&sl.d_lab, sl.lab_pitch * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&sl.d_mask, sl.mask_pitch * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&sl.d_count, 256)) != cudaSuccess) return e;
    const size_t nrm_row = (size_t)W * (c.nrm_bytes_px == 12 ? 4 : 8);
    if (s->cfg.results_to_host) {
        const size_t hb = nrm_row * nrm_rows + (size_t)W * 4 * 3 * H + (size_t)W * 4 * H + (size_t)W * H + 64;
        if ((e = cudaMallocHost(&sl.h_out, hb)) != cudaSuccess) return e;
        char* p = static_cast<char*>(sl.h_out);
        sl.h_nrm = p;
        p += nrm_row * nrm_rows;
        sl.h_pts = reinterpret_cast<float*>(p);
        p += (size_t)W * 4 * 3 * H;
        sl.h_lab = reinterpret_cast<int32_t*>(p);
        p += (size_t)W * 4 * H;
        sl.h_mask = reinterpret_cast<uint8_t*>(p);
        p += (size_t)W * H;
        sl.h_count = reinterpret_cast<int32_t*>(p);
    }
    if ((e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess) return e;

    sn_frame_in fi{sl.d_in, sl.in_pitch};
    sn_frame_out fo{};
    fo.den = nullptr;
    fo.normals = sl.d_nrm;
    fo.normals_pitch = sl.nrm_pitch;
    fo.points = sl.d_pts;
    fo.points_pitch = sl.pts_pitch;
    fo.labels = sl.d_lab;
    fo.labels_pitch = sl.lab_pitch;
    fo.mask = sl.d_mask;
    fo.mask_pitch = sl.mask_pitch;
    fo.num_components = sl.d_count;
    // one eager run (module load, kernel attributes), then capture the graph
    if (sn_run_frame(c.ctx, &fi, &fo, cap) != SN_OK) return cudaErrorUnknown;
    if ((e = cudaStreamSynchronize(cap)) != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    sn_status st = sn_run_frame(c.ctx, &fi, &fo, cap);
    if (st == SN_OK && s->cfg.results_to_host) {
        cudaMemcpy2DAsync(sl.h_nrm, nrm_row, sl.d_nrm, sl.nrm_pitch, nrm_row, nrm_rows, cudaMemcpyDeviceToHost, cap);
        cudaMemcpy2DAsync(sl.h_pts, (size_t)W * 4, sl.d_pts, sl.pts_pitch, (size_t)W * 4, 3 * (size_t)H,
                          cudaMemcpyDeviceToHost, cap);
        cudaMemcpy2DAsync(sl.h_lab, (size_t)W * 4, sl.d_lab, sl.lab_pitch, (size_t)W * 4, H, cudaMemcpyDeviceToHost, cap);
        cudaMemcpy2DAsync(sl.h_mask, (size_t)W, sl.d_mask, sl.mask_pitch, (size_t)W, H, cudaMemcpyDeviceToHost, cap);
        cudaMemcpyAsync(sl.h_count, sl.d_count, 4, cudaMemcpyDeviceToHost, cap);
    }
    e = cudaStreamEndCapture(cap, &graph);
    if (st != SN_OK) return cudaErrorUnknown;
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&sl.exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

void free_slot(Slot& sl) {
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.done) cudaEventDestroy(sl.done);
    cudaFree(sl.d_in);
    cudaFree(sl.d_nrm);
    cudaFree(sl.d_pts);
    cudaFree(sl.d_lab);
    cudaFree(sl.d_mask);
    cudaFree(sl.d_count);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    sl = Slot();
}

// Admits waiting requests, earliest arrival first, into free slots of their
// camera and launches them.  Called with the lock held.
void admit(sn_server* s, std::vector<int>& flying) {
    for (;;) {
        int best = -1;
        double t_best = 0.0;
        int free_slot = -1;
        for (size_t ci = 0; ci < s->cams.size(); ci++) {
            Cam& c = s->cams[ci];
            if (c.queue.empty()) continue;
            int f = -1;
            for (int si : c.slots)
                if (!s->slots[si].busy && !s->slots[si].held) {
                    f = si;
                    break;
                }
            if (f < 0) continue;
            if (best < 0 || c.queue.front().t_arrival < t_best) {
                best = (int)ci;
                t_best = c.queue.front().t_arrival;
                free_slot = f;
            }
        }
        if (best < 0) return;
        Cam& c = s->cams[best];
        Req r = c.queue.front();
        c.queue.pop_front();
        s->waiting--;
        Slot& sl = s->slots[free_slot];
        cudaStream_t st = s->streams[s->rr++ % s->streams.size()];
        cudaError_t e = cudaMemcpy2DAsync(sl.d_in, sl.in_pitch, r.host, r.pitch, (size_t)c.cfg.W * c.in_elem,
                                          c.cfg.H, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, st);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
        if (e != cudaSuccess) {
            s->err = SN_ECUDA;
            continue;
        }
        sl.busy = true;
        sl.sim = r.sim;
        sl.tag = r.tag;
        sl.t_arrival = r.t_arrival;
        s->inflight++;
        flying.push_back(free_slot);
    }
}

void scheduler(sn_server* s) {
    cudaSetDevice(s->device);
    std::vector<int> flying;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && flying.empty()) break;
            if (flying.empty() && s->waiting == 0) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            admit(s, flying);
        }
        // poll the requests in flight; completion time is taken when seen
        bool any = false;
        for (size_t i = 0; i < flying.size();) {
            Slot& sl = s->slots[flying[i]];
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                i++;
                continue;
            }
            const double t = now_s();
            any = true;
            std::lock_guard<std::mutex> lk(s->mu);
            if (q != cudaSuccess) s->err = SN_ECUDA;
            sl.busy = false;
            s->inflight--;
            const Cam& c = s->cams[sl.cam];
            if (sl.sim) {
                s->sim_lat.push_back((t - sl.t_arrival) * 1e3);
                s->sim_done_px += (long long)c.cfg.W * c.cfg.H;
                s->sim_last_done = t;
            } else {
                sn_serve_result r{};
                r.tag = sl.tag;
                r.camera = sl.cam;
                r.slot = flying[i];
                r.latency_ms = (t - sl.t_arrival) * 1e3;
                if (s->cfg.results_to_host) {
                    r.normals = sl.h_nrm;
                    r.points = sl.h_pts;
                    r.labels = sl.h_lab;
                    r.mask = sl.h_mask;
                    r.num_components = *sl.h_count;
                    sl.held = true;
                }
                s->completed.push_back(r);
            }
            flying[i] = flying.back();
            flying.pop_back();
        }
        if (!any) std::this_thread::yield();
    }
}

}  // namespace

extern "C" {

sn_status sn_server_create(const sn_server_config* cfg, sn_server** out) {
    if (!cfg || !out || cfg->n_cameras < 1 || !cfg->cameras || cfg->max_slots_per_camera < 1 || cfg->n_streams < 1 ||
        cfg->n_streams > 16 || cfg->queue_depth < 1)
        return SN_EINVAL;
    *out = nullptr;
    sn_server* s = new sn_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->cams.resize(cfg->n_cameras);
    sn_status st = SN_OK;
    for (int i = 0; i < cfg->n_cameras && st == SN_OK; i++) {
        Cam& c = s->cams[i];
        c.cfg = cfg->cameras[i];
        c.in_elem = c.cfg.params.in_dtype == SN_IN_F32 ? 4 : 2;
        c.nrm_bytes_px = c.cfg.params.normal_fmt == SN_NORMALS_F32X3 ? 12 : 8;
        st = sn_create(&c.cfg.cam, c.cfg.W, c.cfg.H, &c.cfg.params, &c.ctx);
        if (st == SN_OK && c.cfg.params.learned) {
            // the weights go in before the slots' graphs capture the chain
            st = c.cfg.gate_weights ? sn_load_gate_weights(c.ctx, c.cfg.gate_weights, c.cfg.gate_weights_bytes)
                                    : SN_EINVAL;
            c.cfg.gate_weights = nullptr;  // the caller's buffer is not kept
        }
    }
    if (st != SN_OK) {
        sn_server_destroy(s);
        return st;
    }
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        sn_server_destroy(s);
        return SN_ECUDA;
    }
    // slots round-robin over the cameras until the budget is used
    size_t left = cfg->memory_budget;
    bool grew = true;
    for (int k = 0; k < cfg->max_slots_per_camera && grew; k++) {
        grew = false;
        for (int i = 0; i < cfg->n_cameras; i++) {
            Cam& c = s->cams[i];
            const size_t b = slot_bytes(c);
            if (b > left) continue;
            Slot sl;
            sl.cam = i;
            const cudaError_t e = make_slot(s, c, sl, cap);
            if (e != cudaSuccess) {
                free_slot(sl);
                cudaGetLastError();
                continue;
            }
            left -= b;
            c.slots.push_back((int)s->slots.size());
            s->slots.push_back(sl);
            grew = true;
        }
    }
    cudaStreamDestroy(cap);
    for (auto& c : s->cams)
        if (c.slots.empty()) {
            sn_server_destroy(s);
            return SN_ENOMEM;
        }
    s->streams.resize(cfg->n_streams);
    for (auto& st2 : s->streams)
        if (cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking) != cudaSuccess) {
            sn_server_destroy(s);
            return SN_ECUDA;
        }
    s->thread = std::thread(scheduler, s);
    *out = s;
    return SN_OK;
}

sn_status sn_server_destroy(sn_server* s) {
    if (!s) return SN_OK;
    if (s->thread.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            for (auto& c : s->cams) {
                s->waiting -= (long long)c.queue.size();
                c.queue.clear();
            }
        }
        s->cv.notify_all();
        s->thread.join();
    }
    for (auto st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (auto& sl : s->slots) free_slot(sl);
    for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (auto& c : s->cams)
        if (c.ctx) sn_destroy(c.ctx);
    delete s;
    return SN_OK;
}

int sn_server_slots(const sn_server* s, int cam) {
    if (!s || cam < 0 || cam >= (int)s->cams.size()) return -1;
    return (int)s->cams[cam].slots.size();
}

sn_status sn_server_submit(sn_server* s, int cam, const void* host, size_t pitch, uint64_t tag) {
    if (!s || cam < 0 || cam >= (int)s->cams.size() || !host) return SN_EINVAL;
    const Cam& c = s->cams[cam];
    if (pitch < (size_t)c.cfg.W * c.in_elem) return SN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->err != SN_OK) return s->err;
        if ((int)s->cams[cam].queue.size() >= s->cfg.queue_depth) return SN_EBUSY;
        s->cams[cam].queue.push_back(Req{cam, host, pitch, tag, now_s(), false});
        s->waiting++;
    }
    s->cv.notify_one();
    return SN_OK;
}

int sn_server_poll(sn_server* s, sn_serve_result* out, int max) {
    if (!s || !out || max <= 0) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->completed.empty()) {
        out[n++] = s->completed.front();
        s->completed.pop_front();
    }
    return n;
}

sn_status sn_server_release(sn_server* s, int cam, int slot) {
    if (!s || slot < 0 || slot >= (int)s->slots.size() || s->slots[slot].cam != cam) return SN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->slots[slot].held = false;
    }
    s->cv.notify_one();
    return SN_OK;
}

sn_status sn_server_simulate(sn_server* s, const sn_serve_sim* sim, sn_serve_stats* out) {
    if (!s || !sim || !out || !sim->frames || !sim->pool_size || !sim->frame_pitch || sim->duration_s <= 0 ||
        sim->rate_scale <= 0 || sim->max_pool < 1)
        return SN_EINVAL;
    const int nc = (int)s->cams.size();
    for (int c = 0; c < nc; c++)
        if (sim->pool_size[c] < 1 || sim->pool_size[c] > sim->max_pool) return SN_EINVAL;
    struct Arr {
        double t;
        int cam, frame;
    };
    std::vector<Arr> arr;
    std::mt19937_64 rng(sim->seed);
    for (int c = 0; c < nc; c++) {
        const double rate = s->cams[c].cfg.rate_hz * sim->rate_scale;
        if (!(rate > 0)) continue;
        std::exponential_distribution<double> gap(rate);
        double t = gap(rng);
        int k = 0;
        while (t < sim->duration_s) {
            arr.push_back(Arr{t, c, k % sim->pool_size[c]});
            k++;
            t += gap(rng);
        }
    }
    std::sort(arr.begin(), arr.end(), [](const Arr& a, const Arr& b) { return a.t < b.t; });
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->sim_lat.clear();
        s->sim_done_px = 0;
        s->sim_last_done = 0.0;
    }
    long long submitted = 0, refused = 0;
    double offered_px = 0.0;
    const double t0 = now_s() + 0.01;
    for (const Arr& a : arr) {
        const double due = t0 + a.t;
        while (now_s() < due) {
            if (due - now_s() > 2e-4)
                std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        const Cam& c = s->cams[a.cam];
        offered_px += (double)c.cfg.W * c.cfg.H;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if ((int)s->cams[a.cam].queue.size() >= s->cfg.queue_depth) {
                refused++;
                continue;
            }
            s->cams[a.cam].queue.push_back(
                Req{a.cam, sim->frames[(size_t)a.cam * sim->max_pool + a.frame], sim->frame_pitch[a.cam],
                    (uint64_t)submitted, due, true});
            s->waiting++;
            submitted++;
        }
        s->cv.notify_one();
    }
    // drain (bounded)
    const double limit = now_s() + 60.0;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->waiting == 0 && s->inflight == 0) break;
        }
        if (now_s() > limit) return SN_ETIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> lat = s->sim_lat;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, (size_t)(q * (lat.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.5);
    out->p99_ms = pct(0.99);
    out->max_ms = lat.empty() ? 0.0 : lat.back();
    out->submitted = submitted;
    out->completed = (long long)lat.size();
    out->refused = refused;
    out->offered_mpix_s = offered_px / sim->duration_s / 1e6;
    const double span = s->sim_last_done - t0;
    out->sustained_mpix_s = span > 0 ? (double)s->sim_done_px / span / 1e6 : 0.0;
    out->wall_s = now_s() - t0;
    return s->err;
}

sn_status sn_server_check(sn_server* s) {
    if (!s) return SN_EINVAL;
    for (auto st : s->streams) cudaStreamSynchronize(st);
    sn_status r = s->err;
    for (auto& c : s->cams) {
        const sn_status e = sn_check_device(c.ctx, nullptr);
        if (e != SN_OK) r = e;
    }
    return r;
}

}  // extern "C"
