// Stage kernels of the surface-normal chain, one kernel per C-ABI stage:
// denoise, affine + normal, point cloud, and the three passes of the
// connected-component labelling (tile-local union-find in shared memory,
// border merge with global atomics, flatten).
#include "sn_device.cuh"
#include "sn_umma.cuh"

namespace sn {

constexpr int kTW = 32;  // tile width  (one warp per tile row)
constexpr int kTH = 8;   // tile height (8 warps per block)

// ---------------------------------------------------------------- denoise
template <int IN>
__global__ void __launch_bounds__(kTW* kTH)
    k_denoise(const Geo g, const char* __restrict__ disp, size_t dp, float* __restrict__ den,
              size_t denp, uint8_t* __restrict__ mask, size_t mp) {
    extern __shared__ int tile[];
    const int R = g.r_d;
    const int TWR = kTW + 2 * R, THR = kTH + 2 * R;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    load_tile<IN>(tile, TWR, THR, disp, dp, x0 - R, y0 - R, g.W, g.H);
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int* c = tile + (threadIdx.y + R) * TWR + threadIdx.x + R;
    const int Dc = c[0];
    float out = 0.0f;
    uint8_t m = 0;
    if (Dc > 0) {
        bool fit;
        out = denoise_at(c, TWR, R, Dc, g.K_range, fit);
        m = SN_MASK_VALID | (fit ? SN_MASK_DENOISED : 0);
    }
    reinterpret_cast<float*>(reinterpret_cast<char*>(den) + (size_t)y * denp)[x] = out;
    mask[(size_t)y * mp + x] = m;
}

// ---------------------------------------------------------------- affine + normal
template <int IN, int SUP>
__global__ void __launch_bounds__(kTW* kTH)
    k_affine(const Geo g, const __grid_constant__ StarTable T, const char* __restrict__ disp,
             size_t dp, const float* __restrict__ den, size_t denp, char* __restrict__ nrm,
             size_t np, uint8_t* __restrict__ mask, size_t mp, int mask_or) {
    extern __shared__ int tile[];
    // ST needs the edge bit of every pixel a ray can reach: one more halo row
    const int R = SUP == SN_SUPPORT_FIXED ? g.r_a : (SUP == SN_SUPPORT_STARFILL_ST ? g.steps + 1 : g.steps);
    const int TWR = kTW + 2 * R, THR = kTH + 2 * R;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    load_tile<IN>(tile, TWR, THR, disp, dp, x0 - R, y0 - R, g.W, g.H);
    __syncthreads();
    uint8_t* E = reinterpret_cast<uint8_t*>(tile + TWR * THR);  // ST edge bytes, laid out like the tile
    if (SUP == SN_SUPPORT_STARFILL_ST) {
        for (int i = threadIdx.y * kTW + threadIdx.x; i < TWR * THR; i += kTW * kTH) {
            const int ly = i / TWR, lx = i - ly * TWR;
            bool e = true;  // the outer ring is never reached by a ray
            if (lx > 0 && lx < TWR - 1 && ly > 0 && ly < THR - 1)
                e = st_edge(g, tile[i], tile[i - 1], tile[i + 1], tile[i - TWR], tile[i + TWR]);
            E[i] = e;
        }
        __syncthreads();
    }
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const int* c = tile + (threadIdx.y + R) * TWR + threadIdx.x + R;
    const int Dc = c[0];
    float n[3] = {0.0f, 0.0f, 0.0f};
    uint8_t m = 0;
    if (Dc > 0) {
        m = SN_MASK_VALID;
        const float dtil =
            __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(den) + (size_t)y * denp) + x);
        AffSums s;
        if (SUP == SN_SUPPORT_FIXED)
            fixed_support(c, TWR, R, Dc, s);
        else if (SUP == SN_SUPPORT_STARFILL_ST)
            star_support_st(c, E + (c - tile), TWR, Dc, T, g.dirs, g.steps, s);
        else
            star_support(c, TWR, Dc, g.K_cd, T, g.dirs, g.steps, s);
        bool fp64;
        if (solve_normal(s, Dc, dtil, x, y, g, n, fp64)) m |= SN_MASK_NORMAL | (fp64 ? SN_MASK_FP64 : 0);
    }
    if (g.normal_fmt == SN_NORMALS_F32X3) {
        const size_t plane = (size_t)g.H * np;
        float* p0 = reinterpret_cast<float*>(nrm + (size_t)y * np) + x;
        p0[0] = n[0];
        *reinterpret_cast<float*>(reinterpret_cast<char*>(p0) + plane) = n[1];
        *reinterpret_cast<float*>(reinterpret_cast<char*>(p0) + 2 * plane) = n[2];
    } else {
        short4 q;
        q.x = snorm16(n[0]);
        q.y = snorm16(n[1]);
        q.z = snorm16(n[2]);
        q.w = 0;
        reinterpret_cast<short4*>(nrm + (size_t)y * np)[x] = q;
    }
    uint8_t* mo = mask + (size_t)y * mp + x;
    *mo = mask_or ? (uint8_t)(*mo | m) : m;
}

// ---------------------------------------------------------------- points
__global__ void __launch_bounds__(kTW* kTH)
    k_points(const Geo g, const float* __restrict__ den, size_t denp, const uint8_t* __restrict__ mask,
             size_t mp, float* __restrict__ pts, size_t pp) {
    const int x = blockIdx.x * kTW + threadIdx.x, y = blockIdx.y * kTH + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const float d = __ldg(reinterpret_cast<const float*>(reinterpret_cast<const char*>(den) + (size_t)y * denp) + x);
    const uint8_t m = __ldg(mask + (size_t)y * mp + x);
    float X = 0.0f, Y = 0.0f, Z = 0.0f;
    if (m & SN_MASK_VALID) {
        X = g.B * ((float)x - g.cx) / d;
        Y = g.B_fx_over_fy * ((float)y - g.cy) / d;
        Z = g.fxB / d;
    }
    const size_t plane = (size_t)g.H * pp;
    char* p0 = reinterpret_cast<char*>(pts) + (size_t)y * pp + (size_t)x * 4;
    *reinterpret_cast<float*>(p0) = X;
    *reinterpret_cast<float*>(p0 + plane) = Y;
    *reinterpret_cast<float*>(p0 + 2 * plane) = Z;
}

// ---------------------------------------------------------------- components
// Tile-local tiles of kCclTile = 32 columns by kCclTH rows; each warp labels
// kCclRows consecutive rows.
constexpr int kCclTH = 64, kCclRows = 4, kCclWarps = kCclTH / kCclRows;
static_assert(kCclTH % kCclRows == 0 && kCclTile * kCclTH <= 4096, "finds bounded by the tile size");
// Pass 1: union-find inside each 32 x kCclTH tile (shared memory); every pixel
// receives the global index of its tile-local root (the smallest index of
// its tile-local component).
template <int IN>
__global__ void __launch_bounds__(kCclTile * kCclWarps)
    k_ccl_local(const Geo g, const char* __restrict__ disp, size_t dp, int* __restrict__ labels,
                size_t lpe, int* __restrict__ count, const __grid_constant__ CUtensorMap dmap, int use_tma) {
    // Warp w labels rows 4 w .. 4 w + 3 of the 32 x kCclTH tile, lane = column,
    // codes and pair thresholds in registers: the pixels joined to their left
    // neighbour form runs, labelled by the run's first lane (from a ballot of
    // left edges); then vertical edges join the runs of adjacent rows in a
    // shared-memory union-find (an edge implied by its left neighbour's is
    // skipped).  A warp's first row meets the row above through shared memory.
    constexpr int kRows = kCclRows;
    __shared__ int Ls[kCclTile * kCclTH];
    __shared__ int2 Last[kCclWarps][kCclTile];  // (D, t) of each warp's last row
    __shared__ unsigned Lrow[kCclWarps];  // left-edge ballot of each warp's last row
    // the tile's raw disparities by one TMA copy (zero outside the image;
    // the box starts on a 32-element column, a 16-byte boundary)
    constexpr int kES = IN == SN_IN_F32 ? 4 : 2;
    __shared__ __align__(128) unsigned char raw[kCclTile * kCclTH * kES];
    __shared__ uint64_t sbar;
    const int x0 = blockIdx.x * kCclTile, y0 = blockIdx.y * kCclTH;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * kCclTile + lane;
    if (count && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) *count = 0;
    const bool tma = use_tma && (umma::smem_addr(raw) & 127u) == 0;
    // one thread issues the copy and waits for it (sleeping between polls);
    // the block barrier publishes the copy and the outcome (as in stage_tile)
    bool ok = true;
    if (tma) {
        if (tid == 0) {
            umma::mbar_init(&sbar, 1);
            umma::mbar_expect_tx(&sbar, sizeof(raw));
            umma::tma_load_2d(raw, &dmap, x0, y0, &sbar);
            ok = umma::mbar_wait_ns(&sbar, 0, umma::kWaitNs);
            if (!ok) {
                // gave up: report, use no box entry, and wait once more
                // (bounded) for the copy in flight before the CTA can exit
                atomicOr(g.err, kErrMmaWait);
                umma::mbar_wait_ns(&sbar, 0, umma::kDrainNs);
            }
        }
        ok = __syncthreads_and(ok);
    }
    ok = tma && ok;
    // codes and thresholds (pair_thr_v: -1 for an invalid code, so that the
    // pair test needs no validity check)
    int D[kRows], T[kRows];
#pragma unroll
    for (int k = 0; k < kRows; k++) {
        const int r = kRows * w + k, i = r * kCclTile + lane;
        int d = 0;
        if (ok) {
            if constexpr (IN == SN_IN_F32)
                d = code_from_float(reinterpret_cast<const float*>(raw)[i]);
            else if constexpr (IN == SN_IN_F16)
                d = code_from_float(__half2float(reinterpret_cast<const __half*>(raw)[i]));
            else
                d = reinterpret_cast<const unsigned short*>(raw)[i];
        } else if (!tma) {
            d = load_code<IN>(disp, dp, x0 + lane, y0 + r, g.W, g.H);
        }
        D[k] = d;
        T[k] = pair_thr_v(d, g.K_pair);
    }
    Last[w][lane] = make_int2(D[kRows - 1], T[kRows - 1]);
    __syncthreads();
    const unsigned upto = 0xffffffffu >> (31 - lane);
    int run[kRows];
    bool eU[kRows];
    unsigned Lb[kRows], Ub[kRows];
#pragma unroll
    for (int k = 0; k < kRows; k++) {
        const int r = kRows * w + k;
        const int Dl = __shfl_up_sync(0xffffffffu, D[k], 1), Tl = __shfl_up_sync(0xffffffffu, T[k], 1);
        const bool eL = lane > 0 && pair_edge_v(D[k], T[k], Dl, Tl);
        if (k > 0) {
            eU[k] = pair_edge_v(D[k], T[k], D[k - 1], T[k - 1]);
        } else {
            const int2 up = w > 0 ? Last[w - 1][lane] : make_int2(0, -1);
            eU[k] = pair_edge_v(D[k], T[k], up.x, up.y);
        }
        Lb[k] = __ballot_sync(0xffffffffu, eL);
        Ub[k] = __ballot_sync(0xffffffffu, eU[k]);
        run[k] = r * kCclTile + (31 - __clz(~Lb[k] & upto));
        Ls[r * kCclTile + lane] = D[k] > 0 ? run[k] : -1;
    }
    if (lane == 0) Lrow[w] = Lb[kRows - 1];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRows; k++) {
        if (!eU[k]) continue;
        const int r = kRows * w + k;
        const unsigned Lup = k > 0 ? Lb[k - 1] : Lrow[w > 0 ? w - 1 : 0];  // eU[0] is false in row 0
        const bool implied = lane > 0 && ((Ub[k] >> (lane - 1)) & 1u) && ((Lb[k] >> lane) & 1u) && ((Lup >> lane) & 1u);
        if (!implied) union_s(Ls, run[k], (r - 1) * kCclTile + (31 - __clz(~Lup & upto)), g.err);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRows; k++) {
        const int r = kRows * w + k;
        const int x = x0 + lane, y = y0 + r;
        if (x >= g.W || y >= g.H) continue;
        int out = -1;
        if (D[k] > 0) {
            const int root = find_s_halve(Ls, run[k]);
            out = (y0 + root / kCclTile) * g.W + x0 + (root % kCclTile);
        }
        labels[(size_t)y * lpe + x] = out;
    }
}

// Pass 2: join components across tile borders (global atomicMin union).
// Tiles are tw x th pixels.  Row b of the grid takes the vertical border
// x = (b + 1) tw for b < nbx - 1, else the horizontal border
// y = (b - nbx + 2) th; thread s of the row takes the border's 4-neighbour
// pair at row (column) s.  The 32 pairs of a warp lie along one border: of
// the pairs with an edge that join the same two labels only the first
// unites them.
template <int IN>
__global__ void __launch_bounds__(256)
    k_ccl_merge(const Geo g, const char* __restrict__ disp, size_t dp, int* labels, size_t lpe,
                int nbx, int tw, int th) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const bool vertical = b < nbx - 1;
    const int len = vertical ? g.H : g.W;
    if ((int)(blockIdx.x * blockDim.x) >= len) return;  // the whole block lies past the border's end
    const int lane = threadIdx.x & 31;
    int px, py, qx, qy;
    if (vertical) {
        qx = (b + 1) * tw;
        px = qx - 1;
        py = qy = s;
    } else {
        qy = (b - nbx + 2) * th;
        py = qy - 1;
        px = qx = s;
    }
    bool act = s < len;
    int lp = 0, lq = 0;
    unsigned long long key = ~0ull - (unsigned)lane;  // unique for lanes without an edge
    if (act) {
        const int Dp = load_code<IN>(disp, dp, px, py, g.W, g.H);
        const int Dq = load_code<IN>(disp, dp, qx, qy, g.W, g.H);
        act = pair_edge(Dp, Dq, g.K_pair);
        if (act) {
            lp = __ldcg(labels + (size_t)py * lpe + px);
            lq = __ldcg(labels + (size_t)qy * lpe + qx);
            key = ((unsigned long long)(unsigned)lp << 32) | (unsigned)lq;
        }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (act && lp != lq && (int)(__ffs(peers) - 1) == lane) {
        const LabelIndex li{g.W, g.w_rcp, lpe};
        union_g(labels, li, lp, lq, g.err, g.walk_limit);
    }
}

// Pass 3: every pixel points at its global root, which is the smallest
// index of its component; roots are counted.  A thread takes kFlatPix
// pixels of one column of a kTW x kTH tile (their label loads overlap, and
// a label equal to the previous pixel's reuses its root).
constexpr int kFlatPix = 8;
__global__ void __launch_bounds__(kTW * kTH / kFlatPix)
    k_ccl_flatten(const Geo g, int* labels, size_t lpe, int* count) {
    const int x = blockIdx.x * kTW + threadIdx.x;
    const int y0 = blockIdx.y * kTH + threadIdx.y;
    constexpr int kStep = kTH / kFlatPix;
    int l[kFlatPix];
#pragma unroll
    for (int i = 0; i < kFlatPix; i++) {
        const int y = y0 + i * kStep;
        l[i] = (x < g.W && y < g.H) ? __ldcg(labels + (size_t)y * lpe + x) : -1;
    }
    const LabelIndex li{g.W, g.w_rcp, lpe};
    int roots = 0, prev_l = -1, prev_r = -1;
#pragma unroll
    for (int i = 0; i < kFlatPix; i++) {
        if (l[i] < 0) continue;
        const int y = y0 + i * kStep;
        const int r = l[i] == prev_l ? prev_r : find_g(labels, li, l[i], g.err, g.walk_limit);
        prev_l = l[i];
        prev_r = r;
        if (r != l[i]) __stcg(labels + (size_t)y * lpe + x, r);
        roots += r == y * g.W + x;
    }
    if (count && roots) atomicAdd(count, roots);
}

// ---------------------------------------------------------------- the reciprocal of every code
// rcp_approx of D = 1..kDMax as the kernels stage it (+inf for the invalid
// code 0), for the tests that check its error bound.
__global__ void k_rcp_codes(float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= kDMax) out[i] = i == 0 ? __int_as_float(0x7f800000) : rcp_approx((float)i);
}

cudaError_t rcp_codes(float* host_out) {
    float* d = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(float) * (kDMax + 1));
    if (e == cudaSuccess) {
        k_rcp_codes<<<(kDMax + 1 + 255) / 256, 256, 0, st>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, sizeof(float) * (kDMax + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d) cudaFree(d);
    if (st) cudaStreamDestroy(st);
    return e;
}

// ---------------------------------------------------------------- launchers
static dim3 grid2(const Geo& g) { return dim3((g.W + kTW - 1) / kTW, (g.H + kTH - 1) / kTH); }

cudaError_t launch_denoise(const Geo& g, const void* disp, size_t dp, float* den, size_t denp,
                           uint8_t* mask, size_t mp, cudaStream_t s, Marks& mk) {
    if (g.r_d == 2) {
        const cudaError_t e = launch_denoise5(g, disp, dp, den, denp, mask, mp, s);
        mk.after(s);
        return e;
    }
    const int R = g.r_d;
    const size_t smem = sizeof(int) * (kTW + 2 * R) * (kTH + 2 * R);
    const char* d = static_cast<const char*>(disp);
    switch (g.in_dtype) {
        case SN_IN_F32: k_denoise<SN_IN_F32><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, d, dp, den, denp, mask, mp); break;
        case SN_IN_F16: k_denoise<SN_IN_F16><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, d, dp, den, denp, mask, mp); break;
        default: k_denoise<SN_IN_U16X256><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, d, dp, den, denp, mask, mp); break;
    }
    mk.after(s);
    return cudaGetLastError();
}

template <int IN>
static void affine_dispatch(const Geo& g, const StarTable& t, const char* d, size_t dp, const float* den,
                            size_t denp, char* nrm, size_t np, uint8_t* mask, size_t mp, int mor,
                            size_t smem, cudaStream_t s) {
    if (g.support == SN_SUPPORT_FIXED)
        k_affine<IN, SN_SUPPORT_FIXED><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, t, d, dp, den, denp, nrm, np, mask, mp, mor);
    else if (g.support == SN_SUPPORT_STARFILL_ST)
        k_affine<IN, SN_SUPPORT_STARFILL_ST><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, t, d, dp, den, denp, nrm, np, mask, mp, mor);
    else
        k_affine<IN, SN_SUPPORT_STARFILL_CD><<<grid2(g), dim3(kTW, kTH), smem, s>>>(g, t, d, dp, den, denp, nrm, np, mask, mp, mor);
}

cudaError_t launch_affine(const Geo& g, const StarTable& t, const void* disp, size_t dp,
                          const float* den, size_t denp, void* nrm, size_t np, uint8_t* mask,
                          size_t mp, bool mask_or, cudaStream_t s, Marks& mk) {
    if (g.support == SN_SUPPORT_STARFILL_CD && star_is_m8(t, g.dirs, g.steps)) {
        const cudaError_t e = launch_affine_star8(g, disp, dp, den, denp, nrm, np, mask, mp, mask_or, s);
        mk.after(s);
        return e;
    }
    const bool st = g.support == SN_SUPPORT_STARFILL_ST;
    const int R = g.support == SN_SUPPORT_FIXED ? g.r_a : (st ? g.steps + 1 : g.steps);
    // tile ints (+ one edge byte per tile entry for ST); at most 33 KB (s = 30)
    const size_t smem = (sizeof(int) + (st ? 1 : 0)) * (kTW + 2 * R) * (kTH + 2 * R);
    const char* d = static_cast<const char*>(disp);
    char* n = static_cast<char*>(nrm);
    switch (g.in_dtype) {
        case SN_IN_F32: affine_dispatch<SN_IN_F32>(g, t, d, dp, den, denp, n, np, mask, mp, mask_or, smem, s); break;
        case SN_IN_F16: affine_dispatch<SN_IN_F16>(g, t, d, dp, den, denp, n, np, mask, mp, mask_or, smem, s); break;
        default: affine_dispatch<SN_IN_U16X256>(g, t, d, dp, den, denp, n, np, mask, mp, mask_or, smem, s); break;
    }
    mk.after(s);
    return cudaGetLastError();
}

cudaError_t launch_points(const Geo& g, const float* den, size_t denp, const uint8_t* mask, size_t mp,
                          float* pts, size_t pp, cudaStream_t s, Marks& mk) {
    k_points<<<grid2(g), dim3(kTW, kTH), 0, s>>>(g, den, denp, mask, mp, pts, pp);
    mk.after(s);
    return cudaGetLastError();
}

cudaError_t launch_ccl_merge_flatten(const Geo& g, const void* disp, size_t dp, int32_t* labels, size_t lp,
                                     int32_t* count, int tw, int th, cudaStream_t s, Marks& mk) {
    const int nbx = (g.W + tw - 1) / tw, nby = (g.H + th - 1) / th;
    const size_t lpe = lp / sizeof(int32_t);
    const char* d = static_cast<const char*>(disp);
    const int borders = (nbx - 1) + (nby - 1);
    const int longest = g.W > g.H ? g.W : g.H;
    const dim3 mg((unsigned)((longest + 255) / 256), (unsigned)borders);
    if (borders > 0) {
        switch (g.in_dtype) {
            case SN_IN_F32: k_ccl_merge<SN_IN_F32><<<mg, 256, 0, s>>>(g, d, dp, labels, lpe, nbx, tw, th); break;
            case SN_IN_F16: k_ccl_merge<SN_IN_F16><<<mg, 256, 0, s>>>(g, d, dp, labels, lpe, nbx, tw, th); break;
            default: k_ccl_merge<SN_IN_U16X256><<<mg, 256, 0, s>>>(g, d, dp, labels, lpe, nbx, tw, th); break;
        }
    }
    mk.after(s, borders > 0);
    k_ccl_flatten<<<grid2(g), dim3(kTW, kTH / kFlatPix), 0, s>>>(g, labels, lpe, count);
    mk.after(s);
    return cudaGetLastError();
}

cudaError_t launch_components(const Geo& g, const void* disp, size_t dp, int32_t* labels, size_t lp,
                              int32_t* count, cudaStream_t s, Marks& mk) {
    const int nbx = (g.W + kCclTile - 1) / kCclTile, nby = (g.H + kCclTH - 1) / kCclTH;
    const size_t lpe = lp / sizeof(int32_t);
    const char* d = static_cast<const char*>(disp);
    const dim3 lg(nbx, nby), lb(kCclTile, kCclWarps);
    CUtensorMap dmap{};
    const int tma = encode_disp_map(&dmap, disp, dp, g.W, g.H, g.in_dtype, kCclTile, kCclTH) == cudaSuccess;
    switch (g.in_dtype) {
        case SN_IN_F32: k_ccl_local<SN_IN_F32><<<lg, lb, 0, s>>>(g, d, dp, labels, lpe, count, dmap, tma); break;
        case SN_IN_F16: k_ccl_local<SN_IN_F16><<<lg, lb, 0, s>>>(g, d, dp, labels, lpe, count, dmap, tma); break;
        default: k_ccl_local<SN_IN_U16X256><<<lg, lb, 0, s>>>(g, d, dp, labels, lpe, count, dmap, tma); break;
    }
    mk.after(s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_ccl_merge_flatten(g, disp, dp, labels, lp, count, kCclTile, kCclTH, s, mk);
}

}  // namespace sn
