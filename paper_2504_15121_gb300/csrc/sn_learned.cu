// Learned form of the frame kernel (sn_run_frame on a learned context) and
// the gate's probability map (sn_gate_q): two kernels.
//
// k_gate (the network; persistent, two CTAs of 512 threads per SM, 256 TMEM
// columns each) walks its share of the frame's 32 x 16 pixel tiles in a
// software pipeline over two buffers, so that the tensor cores, the TMA
// copies and the CUDA-core phases of different tiles overlap:
//   iteration i:  features of tile i                (CUDA cores)
//                 layer-1 MMAs of tile i             (tensor cores, async)
//                 head of tile i - 1, gate minimum   (CUDA cores)
//                 codes and log2 of tile i + 1       (its TMA copy issued an iteration earlier)
//                 layer-1 epilogue of tile i         (TMEM -> BF16 maps)
//                 layer-2 MMAs of tile i, TMA copy of tile i + 2   (async)
// q is needed only at the lattice points (both coordinates even) within
// SN_LEARNED_RADIUS - 1 of the tile's pixels: 21 x 13 points per tile.
//   * features: per position f0, f1 (FP32 differences of the FP32 log2 of
//     the codes, read from a table, 0 where a code is invalid) and the
//     validity f2; each 16-byte map row holds a position's 4 channels (the
//     fourth zero) and its right neighbour's, in BF16;
//   * layer 1 is an implicit GEMM over every layer-1 position (rows of pitch
//     kP1): K-step dy reads feature row m + dy kP1 as K 0-7 (taps (dy, 0) and
//     (dy, 1)) and row m + dy kP1 + 2 as K 8-15 (tap (dy, 2); the fourth
//     position weighted zero), the second K core matrix 32 bytes on: 3
//     tcgen05.mma (M = 128, N = 16, K = 16, BF16 in, FP32 in TMEM) per
//     128-row tile;
//   * its epilogue (tcgen05.ld; biases in packed FP32 pairs, ReLU and BF16
//     rounding in one instruction) writes the layer-1 map split by the parity
//     of the row and of the column into four planes of pitch kPJ, so that
//     for lattice output (a, b) tap (dy, dx) reads plane (dy % 2, dx % 2) at
//     (a + dy / 2, b + dx / 2): a constant shift per tap, and layer 2 runs as
//     an implicit GEMM over the lattice points only (9 MMAs per 128 points);
//   * head: ReLU as a max with -b2 (b2 folded into the head's constant), a
//     packed FP32 dot product, the sigmoid;
//   * output: the gate bit (minimum of q over the pixel's lattice points
//     >= tau) as SN_MASK_LEARNED in the frame's mask buffer, or q (sn_gate_q).
// k_learned (the chain; 32 x 16 tiles, 256 threads of two pixels each, four
// CTAs per SM: short CTAs hide its barriers better than 512 threads at two
// per SM, although the star walk of the uncertified pixels then spills a
// few registers) stages the tile and
// a halo of 10 by TMA as (D, 1/D), reads the gate bits, and fits certified
// valid pixels on the full 13 x 13 affine and the un-gated 5 x 5 denoise
// window: a row pass per entry (count + 2^16 sum u of the valid samples, sum
// u^2, sum D, sum u D over 13 and 5 columns) and a column pass per pixel
// (weights 1, v, v^2 on the packed word give five moments in three integer
// operations).  The other valid pixels are compacted into a list and take
// the plain chain (range-gated denoise, covered-depth star).
#include <atomic>
#include <mutex>

#include "sn_pixel.cuh"

namespace sn {

namespace {

// ---------------------------------------------------------------- gate kernel geometry (32 x 16 tiles)
// Tile at (x0, y0), both even.  The lattice points within kLatM of a tile
// pixel are x0 - kLatO + 2 b (b < kLatW) by y0 - kLatO + 2 a (a < kLatH).
// Layer 1 is needed one position around them (kH1W x kH1H from x0 - kLatO - 1),
// the features one more (kFW x kFH from x0 - kLatO - 2), the codes one more
// to the right and below (each feature reads its right and lower neighbour).
constexpr int kFastR = SN_LEARNED_RADIUS, kLatM = kFastR - 1;
constexpr int kLatO = kLatM / 2 * 2;                       // largest even offset <= kLatM
constexpr int kLatW = (kTW - 1 + kLatM + kLatO) / 2 + 1;    // 21
constexpr int kLatH = (kTH - 1 + kLatM + kLatO) / 2 + 1;    // 13
constexpr int kH1W = 2 * (kLatW - 1) + 3, kH1H = 2 * (kLatH - 1) + 3;  // 43 x 27
constexpr int kFW = kH1W + 2, kFH = kH1H + 2;              // 45 x 29
constexpr int kLW = kFW + 1, kLH = kFH + 1, kLN = kLW * kLH;  // 46 x 30 codes
constexpr int kP1 = kFW;                                   // row pitch of the feature map and layer 1
constexpr int kMT1 = (kH1H * kP1 + 127) / 128;             // layer-1 MMA tiles
constexpr int kPJ = (kH1W + 1) / 2;                        // pitch of the parity planes
constexpr int kMT2 = (kLatH * kPJ + 127) / 128;            // layer-2 MMA tiles
// feature rows layer 1 reads (the last tile's rows + 2 kP1 + 2), plane
// positions layer 2 reads (the last tile's rows + kPJ + 1)
constexpr int kFeatN = kFW * kFH;
constexpr int kFeatPos = (kMT1 * 128 + 2 * kP1 + 2 + 7) & ~7;
constexpr int kPlanePos = (kMT2 * 128 + kPJ + 1 + 7) & ~7;
static_assert(kLatO >= 2 && kLatO % 2 == 0 && kLatO <= kLatM, "lattice origin");
static_assert(kMT2 <= kThreads / 128, "one layer-2 tile per warp group in the head");
static_assert(((kH1H + 1) / 2 - 1) * kPJ + (kH1W + 1) / 2 - 1 < kPlanePos, "the layer-1 map fits its planes");
constexpr uint32_t kNetIdesc = umma::idesc_bf16<128, 16>();

// The TMA box of one tile: columns x0 - kGX .. x0 - kGX + kGBW - 1 (x0 - kGX
// a multiple of 8 elements, a 16-byte boundary for 4- and 2-byte input),
// rows from y0 - kLatO - 2, kLH of them; code column lx is box column
// lx + kGX - kLatO - 2.
constexpr int kGX = 8, kGBW = 48, kGBH = kLH;
static_assert(kGX >= kLatO + 2 && kGX - kLatO - 2 + kLW <= kGBW && kGBW % 8 == 0, "box covers the codes");
constexpr int kLPerThread = (kLH + kThreads / kLW - 1) / (kThreads / kLW);  // code rows per thread
constexpr size_t kGRawBytes = (size_t)kGBW * kGBH * 4;  // FP32 input; 16-bit input uses half
// One buffer of each map suffices: the features of tile i + 1 are written
// after layer 1 of tile i has completed, its layer-1 map after layer 2 of tile
// i has completed, its codes' log2 after the features of tile i are made.
// TMEM: layer 1's accumulators in columns [0, 16 kMT1), layer 2's in
// [kT2Col, kT2Col + 16 kMT2), so that layer 1 of tile i + 1 runs while the
// head of tile i reads layer 2's.
constexpr uint32_t kT2Col = 16 * kMT1;
static_assert(kT2Col + 16 * kMT2 <= 256, "both layers' accumulators in 256 TMEM columns");
constexpr size_t kGOffRaw = 0;
constexpr size_t kGOffL = kGOffRaw + align128z(kGRawBytes);
constexpr size_t kGOffFeat = kGOffL + align128z(sizeof(float) * kLN);
constexpr size_t kGOffH1 = kGOffFeat + align128z(16 * (size_t)kFeatPos);  // 4 parity planes x 2 channel halves
constexpr size_t kGOffQ = kGOffH1 + align128z(8 * 16 * (size_t)kPlanePos);
constexpr size_t kGOffQRow = kGOffQ + align128z(sizeof(float) * kLatW * kLatH);
constexpr size_t kGOffPar = kGOffQRow + align128z(sizeof(float) * kLatH * kTW);
constexpr size_t kGOffBar = align16z(kGOffPar + kNetImageBytes);  // wbar, tbar, l1, l2, TMEM slot
constexpr size_t kGSmem = align128z(kGOffBar + 8 * 8);
static_assert(2 * (kGSmem + 1024) <= 228 * 1024, "two gate CTAs per SM");
static_assert(kNetImageBytes % 16 == 0 && kGOffPar % 16 == 0, "bulk copy of the weights image");

// ---------------------------------------------------------------- chain kernel layout
constexpr int kLR = 10;                                     // staged halo (the star's reach)
constexpr int kLTWR = kTW + 2 * kLR, kLTHR = kTH + 2 * kLR;  // 52 x 36 staged entries
constexpr int kTileN = kLTWR * kLTHR;
constexpr int kRSRows = kTH + 2 * kFastR;  // row-sum rows: tile rows -kFastR .. kTH - 1 + kFastR
constexpr int kRS = kRSRows * kTW;
static_assert(kFastR <= kLR, "the full window lies in the staged tile");
// tile, then the row sums (the raw TMA box lies where the row sums go: they
// are written after the conversion), the work list, its counter
constexpr size_t kCOffTile = 0;
constexpr size_t kCOffRS = align128z(sizeof(int2) * kTileN);
constexpr size_t kCOffRS5 = kCOffRS + 16 * (size_t)kRS;
constexpr size_t kCOffList = kCOffRS5 + 16 * (size_t)kRS;
constexpr size_t kCOffCnt = kCOffList + sizeof(int) * kThreads;  // room for every pixel of the tile
constexpr size_t kCSmem = align128z(kCOffCnt + 16);
static_assert(tma_bw<SN_IN_F32, kLR, kLTWR>() * kLTHR * 4 + 8 <= 2 * 16 * kRS, "raw box inside the row sums");
// 32 x 8 threads, two pixels each (tile rows ty and ty + 8), four CTAs per SM
constexpr int kCThreads = kTW * 8;
static_assert(kTH == 16, "two pixel rows per thread");
static_assert(4 * (kCSmem + 1024) <= 228 * 1024, "four chain CTAs per SM");

// log2 of every code (FP32, correctly rounded from the FP64 value; NaN for
// code 0, the invalid pixel), read by the features of the inference and the
// training kernels.  Filled once per device.
__device__ float g_log2tab[kDMax + 1];

__global__ void k_log2tab() {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= kDMax) g_log2tab[i] = i == 0 ? __int_as_float(0x7fc00000) : __double2float_rn(log2((double)i));
}

// ---------------------------------------------------------------- small helpers

// BF16 pair (lo = relu(a), hi = relu(b)), rounded to nearest even
__device__ __forceinline__ unsigned relu_bf16x2(float a, float b) {
    unsigned r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// BF16 pair (lo = a, hi = b), rounded to nearest even
__device__ __forceinline__ unsigned bf16x2(float a, float b) {
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// x with NaN replaced by 0 (x itself otherwise: one of the two terms is 0)
__device__ __forceinline__ float nan_to_zero(float x) { return fmaxf(x, 0.0f) + fminf(x, 0.0f); }

template <int IN>
__device__ __forceinline__ int box_code(const unsigned char* raw, int i) {
    if constexpr (IN == SN_IN_F32)
        return code_from_float(reinterpret_cast<const float*>(raw)[i]);
    else if constexpr (IN == SN_IN_F16)
        return code_from_float(__half2float(reinterpret_cast<const __half*>(raw)[i]));
    else
        return reinterpret_cast<const unsigned short*>(raw)[i];
}

// ---------------------------------------------------------------- the weights image
// The B operands: element (n, k) of K-step s at s 512 + (k / 8) 256 +
// (n / 8) 128 + (n % 8) 16 + (k % 8) 2 bytes (16 x 16 BF16 in 8 x 16-byte
// core matrices).  Layer 1, K-step dy: k 0-7 weigh the feature row of
// position dx = 0 (its channels 0-3) and its right neighbour dx = 1 (4-7),
// k 8-15 positions dx = 2 and dx = 3 (zero); channel 3 of a position is
// zero.  Layer 2, K-step tap: k = channel of the layer-1 map.
__global__ void k_net_image(const GateView gv, unsigned char* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned char* W1s = img;
    unsigned char* W2s = img + 3 * 512;
    if (i < 16 * 48) {
        // W1g is [16][80] with k = tap * 8 + channel (tap = 3 dy + dx)
        const int nn = i / 48, k = i % 48;
        const int dy = k / 16, kk = k % 16, dx = 2 * (kk / 8) + ((kk % 8) >= 4), ch = kk % 4;
        *reinterpret_cast<__nv_bfloat16*>(W1s + dy * 512 + (kk / 8) * 256 + (nn / 8) * 128 + (nn % 8) * 16 +
                                          (kk % 8) * 2) =
            (dx <= 2 && ch < 3) ? gv.W1g[nn * 80 + (3 * dy + dx) * 8 + ch] : __float2bfloat16(0.0f);
    }
    if (i < 16 * 144) {
        // W2g is [16][144] with k = tap * 16 + channel
        const int nn = i / 144, k = i % 144, tap = k / 16, ch = k % 16;
        *reinterpret_cast<__nv_bfloat16*>(W2s + tap * 512 + (ch / 8) * 256 + (nn / 8) * 128 + (nn % 8) * 16 +
                                          (ch % 8) * 2) = gv.W2g[i];
    }
}

// ---------------------------------------------------------------- the gate kernel
// QMAP: write q at the pixels with both coordinates even (NaN at the others)
// to qout; otherwise the gate bit into o.mask.
template <int IN, bool QMAP>
__global__ void __launch_bounds__(kThreads, 2)
    k_gate(const Geo g, const FrameOut o, const GateView gv, float* __restrict__ qout, size_t qp,
           const __grid_constant__ CUtensorMap dmap) {
    extern __shared__ __align__(128) unsigned char smem[];
    const unsigned char* W1s = smem + kGOffPar;
    const unsigned char* W2s = W1s + 3 * 512;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kGOffBar);
    uint64_t* wbar = bars;       // the weights copy
    uint64_t* tbar = bars + 1;   // the TMA box (one per tile, in order)
    uint64_t* l1bar = bars + 2;  // layer-1 MMAs (one phase per tile)
    uint64_t* l2bar = bars + 3;  // layer-2 MMAs (one phase per tile)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    unsigned char* raw = smem + kGOffRaw;
    float* qs = reinterpret_cast<float*>(smem + kGOffQ);
    float* qrow = reinterpret_cast<float*>(smem + kGOffQRow);
    const int lane = threadIdx.x, row = threadIdx.y;
    const int tid = row * kTW + lane, warp = tid >> 5;
    const int tilesX = (g.W + kTW - 1) / kTW, tilesY = (g.H + kTH - 1) / kTH;
    const int ntiles = tilesX * tilesY;
    const int n = ((int)blockIdx.x < ntiles) ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    constexpr uint32_t kRawBytes = (uint32_t)kGBW * kGBH * (IN == SN_IN_F32 ? 4 : 2);
    float* L = reinterpret_cast<float*>(smem + kGOffL);
    uint4* feat = reinterpret_cast<uint4*>(smem + kGOffFeat);
    // parity plane p = 2 (row parity) + column parity, channel half h: kPlanePos positions
    auto plane = [&](int p, int h) { return reinterpret_cast<uint4*>(smem + kGOffH1) + (size_t)(2 * p + h) * kPlanePos; };
    auto tile_xy = [&](int i, int& x0, int& y0) {
        const int k = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (k % tilesX) * kTW;
        y0 = (k / tilesX) * kTH;
    };
    auto issue_tma = [&](int i) {
        int x0, y0;
        tile_xy(i, x0, y0);
        umma::mbar_expect_tx(tbar, kRawBytes);
        umma::tma_load_2d(raw, &dmap, x0 - kGX, y0 - kLatO - 2, tbar);
    };
    // counts of what has been put in flight (for the drain; tid 0's view)
    int nt = 0, n1 = 0, n2 = 0;

    if (warp == 0) umma::tmem_alloc(tslot, 256);
    if (tid == 0) {
        umma::mbar_init(wbar, 1);
        umma::mbar_init(tbar, 1);
        umma::mbar_init(l1bar, kMT1);  // one commit per issuing warp
        umma::mbar_init(l2bar, kMT2);
        umma::mbar_expect_tx(wbar, kNetImageBytes);
        umma::bulk_g2s(smem + kGOffPar, gv.net, kNetImageBytes, wbar);
        if (n > 0) {
            issue_tma(0);
            nt++;
        }
    }
    // map positions that no output reads stay zero (they feed dropped GEMM rows)
    for (int i = kFeatN + tid; i < kFeatPos; i += kThreads) feat[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < 8 * kPlanePos; i += kThreads) plane(0, 0)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();  // barriers initialised, TMEM address written
    const uint32_t tmem = *tslot;
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;  // the TMEM lanes this warp may read
    // One thread waits for an asynchronous step (sleeping between polls);
    // the block barrier that follows publishes it and the outcome.
    auto wait1 = [&](uint64_t* bar, int parity) {
        return tid != 0 || umma::mbar_wait_ns(bar, parity, umma::kWaitNs);
    };
    bool ok = wait1(wbar, 0);

    // codes and their log2 of tile i's box into L buffer i & 1 (this
    // thread's entries in registers first, so that the table reads overlap)
    constexpr int kLRowsPerPass = kThreads / kLW;
    static_assert(kLPerThread * kLRowsPerPass >= kLH, "the code region in kLPerThread passes");
    const int lx = tid % kLW, ly0 = tid / kLW;
    const bool lthread = tid < kLRowsPerPass * kLW;
    float Lreg[kLPerThread];
    auto load_L = [&](int i) {  // after the block barrier that follows wait1(tbar, i & 1)
#pragma unroll
        for (int k = 0; k < kLPerThread; k++) {
            const int ly = ly0 + k * kLRowsPerPass;
            if (lthread && ly < kLH) {
                const int D = ok ? box_code<IN>(raw, ly * kGBW + lx + kGX - kLatO - 2) : 0;
                Lreg[k] = __ldg(gv.log2tab + D);
            }
        }
    };
    auto store_L = [&]() {
#pragma unroll
        for (int k = 0; k < kLPerThread; k++) {
            const int ly = ly0 + k * kLRowsPerPass;
            if (lthread && ly < kLH) L[ly * kLW + lx] = Lreg[k];
        }
    };
    // head of tile i (layer 2's accumulators, lattice rows), then the output
    auto head = [&](int i) {
        ok = __syncthreads_and(ok && wait1(l2bar, i & 1));
        umma::fence_after();
        const int t = warp >> 2;
        if (ok && t < kMT2) {
            uint32_t r[16];
            umma::ld16(tmem + kT2Col + tlane + 16 * t, r);
            umma::wait_ld();
            // W3 . relu(acc + b2) + b3 = W3 . max(acc, -b2) + c3 (constants from the kernel parameters)
            float s0 = gv.k.c3, s1 = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                s0 = fmaf(gv.k.w3[2 * c], fmaxf(__uint_as_float(r[2 * c]), gv.k.nb2[2 * c]), s0);
                s1 = fmaf(gv.k.w3[2 * c + 1], fmaxf(__uint_as_float(r[2 * c + 1]), gv.k.nb2[2 * c + 1]), s1);
            }
            const int j = 128 * t + (warp & 3) * 32 + lane, a = j / kPJ, bb = j - a * kPJ;
            if (a < kLatH && bb < kLatW) qs[a * kLatW + bb] = __fdividef(1.0f, 1.0f + __expf(-(s0 + s1)));
        }
        umma::fence_before();
        __syncthreads();
        int x0, y0;
        tile_xy(i, x0, y0);
        const int x = x0 + lane, y = y0 + row;
        const bool inside = x < g.W && y < g.H;
        if constexpr (QMAP) {
            if (inside) {
                float v = __int_as_float(0x7fc00000);
                if (ok && ((lane | row) & 1) == 0) v = qs[((row + kLatO) >> 1) * kLatW + ((lane + kLatO) >> 1)];
                reinterpret_cast<float*>(reinterpret_cast<char*>(qout) + (size_t)y * qp)[x] = v;
            }
        } else {
            // lattice columns b of tile column c: |x0 - kLatO + 2 b - (x0 + c)| <= kLatM,
            // i.e. b from lo(c) = (c - kLatM + kLatO + 1) >> 1, kLatM (c even) or
            // kLatM + 1 (c odd) of them (kLatM odd, kLatO even); the last one is
            // read for every c (in range) and kept only for odd c
            static_assert(kLatM % 2 == 1 && ((kTW - 1 - kLatM + kLatO + 1) >> 1) + kLatM < kLatW &&
                              ((kTH - 1 - kLatM + kLatO + 1) >> 1) + kLatM < kLatH,
                          "lattice window of kLatM or kLatM + 1 points");
            for (int e = tid; e < kLatH * kTW; e += kThreads) {
                const int a = e / kTW, c = e - a * kTW;
                const float* q0 = qs + a * kLatW + ((c - kLatM + kLatO + 1) >> 1);
                float m = q0[0];
#pragma unroll
                for (int k = 1; k < kLatM; k++) m = fminf(m, q0[k]);
                const float last = q0[kLatM];
                qrow[e] = (c & 1) ? fminf(m, last) : m;
            }
            __syncthreads();
            if (inside) {
                const float* q1 = qrow + ((row - kLatM + kLatO + 1) >> 1) * kTW + lane;
                float m = q1[0];
#pragma unroll
                for (int k = 1; k < kLatM; k++) m = fminf(m, q1[k * kTW]);
                const float last = q1[kLatM * kTW];
                if (row & 1) m = fminf(m, last);
                o.mask[(size_t)y * o.mp + x] = (ok && m >= gv.tau) ? (uint8_t)SN_MASK_LEARNED : (uint8_t)0;
            }
        }
    };

    ok = __syncthreads_and(ok && (n == 0 || wait1(tbar, 0)));
    if (n > 0) {
        load_L(0);
        store_L();
    }
    ok = __syncthreads_and(ok);  // the box of tile 0 is read: it may be overwritten
    if (ok && n > 1 && tid == 0) {
        issue_tma(1);
        nt++;
    }
    int i = 0;
    for (; ok && i < n; i++) {
        // ---- features of tile i: each map row holds a position's channels
        // (f0, f1, f2, 0) and its right neighbour's
        {
            uint4* F = feat;
            constexpr int kRowsPerPass = kThreads / kFW;
            constexpr int kPasses = (kFH + kRowsPerPass - 1) / kRowsPerPass;
            // the right neighbour's entries of the last map column read one
            // code past the row, which the code region holds (kLW = kFW + 1,
            // kLH = kFH + 1), and are then zeroed
            static_assert(kLW == kFW + 1 && kLH == kFH + 1, "codes one past the map");
            const int fx = tid % kFW, fy0 = tid / kFW;
            const bool has_right = fx + 1 < kFW;
            if (tid < kRowsPerPass * kFW) {
#pragma unroll
                for (int k = 0; k < kPasses; k++) {
                    const int fy = fy0 + k * kRowsPerPass;
                    if (fy < kFH) {
                        const int e = fy * kLW + fx;
                        const float Lc = L[e], Lr = L[e + 1];
                        uint4 v;
                        v.x = bf16x2(nan_to_zero(Lr - Lc), nan_to_zero(L[e + kLW] - Lc));
                        v.y = Lc == Lc ? 0x3F80u : 0u;  // BF16 1.0 where the code is valid
                        const unsigned z = bf16x2(nan_to_zero(L[e + 2] - Lr), nan_to_zero(L[e + kLW + 1] - Lr));
                        v.z = has_right ? z : 0u;
                        v.w = has_right && Lr == Lr ? 0x3F80u : 0u;
                        F[fy * kFW + fx] = v;
                    }
                }
            }
        }
        umma::fence_proxy_async();
        umma::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        umma::fence_after();
        // ---- layer-1 MMAs of tile i (async; lane 0 of warp t issues MMA
        // tile t), then the head of tile i - 1
        if (lane == 0 && warp < kMT1) {
            const uint64_t bd = umma::desc(umma::smem_addr(W1s), 256, 128);
            const uint64_t a0 = umma::desc(umma::smem_addr(feat + 128 * warp), 32, 128);
#pragma unroll
            for (int dy = 0; dy < 3; dy++)
                umma::mma<kNetIdesc>(tmem + 16 * warp, a0 + dy * kP1, bd + 32 * dy, dy > 0);
            umma::commit(l1bar);
        }
        if (tid == 0) n1++;
        if (i > 0) head(i - 1);
        // ---- codes and log2 of tile i + 1 (in registers), the layer-1
        // epilogue of tile i, then the log2 into their buffer
        ok = __syncthreads_and(ok && (i + 1 >= n || wait1(tbar, (i + 1) & 1)) && wait1(l1bar, i & 1));
        umma::fence_after();
        if (ok && i + 1 < n) load_L(i + 1);
        if (ok) {
#pragma unroll
            for (int k = 0; k < (kMT1 + kThreads / 128 - 1) / (kThreads / 128); k++) {
                const int t = (warp >> 2) + k * (kThreads / 128);
                if (t >= kMT1) break;  // warp-uniform
                uint32_t r[16];
                umma::ld16(tmem + tlane + 16 * t, r);
                umma::wait_ld();
                const int j = 128 * t + (warp & 3) * 32 + lane, hy = j / kP1, hx = j - hy * kP1;
                if (hy < kH1H && hx < kH1W) {
                    unsigned w[8];
#pragma unroll
                    for (int c = 0; c < 8; c++)
                        w[c] = relu_bf16x2(__uint_as_float(r[2 * c]) + gv.k.b1[2 * c],
                                           __uint_as_float(r[2 * c + 1]) + gv.k.b1[2 * c + 1]);
                    const int p = 2 * (hy & 1) + (hx & 1), k = (hy >> 1) * kPJ + (hx >> 1);
                    plane(p, 0)[k] = make_uint4(w[0], w[1], w[2], w[3]);
                    plane(p, 1)[k] = make_uint4(w[4], w[5], w[6], w[7]);
                }
            }
        }
        if (i + 1 < n) store_L();
        umma::fence_proxy_async();
        umma::fence_before();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        umma::fence_after();
        // ---- layer-2 MMAs of tile i on its lattice points (async; lane 0 of
        // warp t issues MMA tile t); the box of tile i + 2 (the one of tile
        // i + 1 has been read)
        if (lane == 0 && warp < kMT2) {
            const uint64_t bd = umma::desc(umma::smem_addr(W2s), 256, 128);
#pragma unroll
            for (int tap = 0; tap < 9; tap++) {
                const int dy = tap / 3, dx = tap % 3;
                const uint64_t a = umma::desc(umma::smem_addr(plane(2 * (dy & 1) + (dx & 1), 0) + 128 * warp),
                                              16 * kPlanePos, 128) +
                                   (dy >> 1) * kPJ + (dx >> 1);
                umma::mma<kNetIdesc>(tmem + kT2Col + 16 * warp, a, bd + 32 * tap, tap > 0);
            }
            umma::commit(l2bar);
        }
        if (tid == 0) {
            n2++;
            if (i + 2 < n) {
                issue_tma(i + 2);
                nt++;
            }
        }
    }
    if (ok && n > 0) head(n - 1);
    ok = __syncthreads_and(ok);
    if (!ok) {
        // Gave up on a wait: record it, and let everything this CTA put in
        // flight drain (bounded) before the TMEM is freed and the CTA exits.
        if (tid == 0) {
            atomicOr(g.err, kErrMmaWait);
            if (nt) umma::mbar_wait_ns(tbar, (nt - 1) & 1, umma::kDrainNs);
            if (n1) umma::mbar_wait_ns(l1bar, (n1 - 1) & 1, umma::kDrainNs);
            if (n2) umma::mbar_wait_ns(l2bar, (n2 - 1) & 1, umma::kDrainNs);
            umma::mbar_wait_ns(wbar, 0, umma::kDrainNs);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after();
        umma::tmem_dealloc(tmem, 256);
    }
}

// ---------------------------------------------------------------- the chain kernel
template <int IN>
__global__ void __launch_bounds__(kCThreads, 4)
    k_learned(const Geo g, const char* __restrict__ disp, size_t dp, const FrameOut o,
              const __grid_constant__ CUtensorMap dmap) {
    extern __shared__ __align__(128) unsigned char smem[];
    int2* tile = reinterpret_cast<int2*>(smem + kCOffTile);
    int4* rs = reinterpret_cast<int4*>(smem + kCOffRS);
    int4* rs5 = reinterpret_cast<int4*>(smem + kCOffRS5);
    int* list = reinterpret_cast<int*>(smem + kCOffList);
    int* cnt = reinterpret_cast<int*>(smem + kCOffCnt);
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTW + lane;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const int x = x0 + lane;
    // the gate bits the gate kernel left in the mask, for rows ty and ty + 8
    // (bit k of cand: row ty + 8 k)
    unsigned cand = 0u;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int y = y0 + ty + 8 * k;
        if (x < g.W && y < g.H && (o.mask[(size_t)y * o.mp + x] & SN_MASK_LEARNED)) cand |= 1u << k;
    }
    if (tid == 0) *cnt = 0;
    stage_tile<IN, kLR, kTH, kCThreads, false>(tile, smem + kCOffRS, &dmap, true, disp, dp, x0, y0, g, kStageRcp);
    // the centre codes (0 outside the image): gated = certified and valid
    auto centre = [&](int k) { return tile[(ty + 8 * k + kLR) * kLTWR + lane + kLR].x; };
    unsigned gated = 0u;
#pragma unroll
    for (int k = 0; k < 2; k++)
        if ((cand >> k & 1u) && centre(k) > 0) gated |= 1u << k;
    if (__syncthreads_or(gated != 0u)) {
        // ---- row pass: for every entry (tile rows -kFastR .. kTH - 1 + kFastR)
        // over |u| <= 2 and |u| <= kFastR: (count + 2^16 sum u) of the valid
        // samples, their sum u^2, the sums of D and of u D (D = 0 where invalid)
#pragma unroll 1
        for (int pass = 0; pass < (kRS + kCThreads - 1) / kCThreads; pass++) {
            const int e = tid + pass * kCThreads;
            if (kRS % kCThreads != 0 && e >= kRS) break;
            const int2* p = tile + (e / kTW + kLR - kFastR) * kLTWR + e % kTW + kLR;
            int A = 0, B = 0, Q0 = 0, Q1 = 0;
#pragma unroll
            for (int u = -2; u <= 2; u++) {
                const int D = p[u].x, v = min(D, 1);
                A += v * (1 + u * 65536);
                B += v * (u * u);
                Q0 += D;
                Q1 += u * D;
            }
            rs5[e] = make_int4(A, B, Q0, Q1);
#pragma unroll
            for (int k = 3; k <= kFastR; k++) {
#pragma unroll
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int u = sgn * k;
                    const int D = p[u].x, v = min(D, 1);
                    A += v * (1 + u * 65536);
                    B += v * (u * u);
                    Q0 += D;
                    Q1 += u * D;
                }
            }
            rs[e] = make_int4(A, B, Q0, Q1);
        }
        __syncthreads();
    }
#pragma unroll 1
    for (int k = 0; k < 2; k++) {
        const int row = ty + 8 * k, y = y0 + row;
        if (gated >> k & 1u) {
            // ---- column pass over 2 kFastR + 1 and 5 rows: with P = count +
            // 2^16 sum u per row, sum P = n + 2^16 Su, sum v P = Sv + 2^16 Suv,
            // sum v^2 P = Svv + 2^16 (sum v^2 u), each low field within 16 bits
            int SA = 0, SAv = 0, SAv2 = 0, SB = 0, SQ1 = 0, SQ0v = 0;
#pragma unroll
            for (int j = -kFastR; j <= kFastR; j++) {
                const int4 a = rs[(row + kFastR + j) * kTW + lane];
                SA += a.x;
                SAv += j * a.x;
                SAv2 += (j * j) * a.x;
                SB += a.y;
                SQ1 += a.w;
                SQ0v += j * a.z;
            }
            int TA = 0, TAv = 0, TAv2 = 0, TB = 0, TQ0 = 0, TQ0v = 0, TQ1 = 0;
#pragma unroll
            for (int j = -2; j <= 2; j++) {
                const int4 a = rs5[(row + kFastR + j) * kTW + lane];
                TA += a.x;
                TAv += j * a.x;
                TAv2 += (j * j) * a.x;
                TB += a.y;
                TQ0 += a.z;
                TQ0v += j * a.z;
                TQ1 += a.w;
            }
            WinSums wa, w2;
            wa.n = SA & 0xFFFF;
            wa.Su = (SA - wa.n) >> 16;
            wa.Sv = (int)(short)(SAv & 0xFFFF);
            wa.Suv = (SAv - wa.Sv) >> 16;
            wa.Svv = SAv2 & 0xFFFF;
            wa.Suu = SB;
            wa.SD = 0;  // not used by the affine fit
            wa.SuD = SQ1;
            wa.SvD = SQ0v;
            w2.n = TA & 0xFFFF;
            w2.Su = (TA - w2.n) >> 16;
            w2.Sv = (int)(short)(TAv & 0xFFFF);
            w2.Suv = (TAv - w2.Sv) >> 16;
            w2.Svv = TAv2 & 0xFFFF;
            w2.Suu = TB;
            w2.SD = TQ0;
            w2.SuD = TQ1;
            w2.SvD = TQ0v;
            PixOut r;
            fast_pixel(g, centre(k), w2, wa, x, y, r);
            emit(g, o, x, y, r);
        } else if (x < g.W && y < g.H && centre(k) <= 0) {
            PixOut r;
            pix_zero(r);
            emit(g, o, x, y, r);
        }
    }
    // ---- the uncertified valid pixels, compacted so that whole warps walk star rays
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int y = y0 + ty + 8 * k;
        const bool need = x < g.W && y < g.H && centre(k) > 0 && !(gated >> k & 1u);
        const unsigned m = __ballot_sync(0xffffffffu, need);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(cnt, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (need) list[base + __popc(m & ((1u << lane) - 1u))] = (ty + 8 * k) * kTW + lane;
    }
    __syncthreads();
    const int nl = *cnt;
    for (int i = tid; i < nl; i += kCThreads) {
        const int p = list[i];
        const int px = p % kTW, py = p / kTW;
        PixOut r;
        plain_pixel<2, kLR, 2, kF64Inline>(g, nullptr, tile + (py + kLR) * kLTWR + px + kLR, kLTWR, x0 + px, y0 + py, r);
        emit(g, o, x0 + px, y0 + py, r);
    }
}

int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int v = cached[dev].load();
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
        cached[dev].store(v);
    }
    return v;
}

template <int IN, bool QMAP>
cudaError_t launch_gate(const Geo& g, const void* disp, size_t dp, const FrameOut& o, const GateView& gv, float* q,
                        size_t qp, cudaStream_t s) {
    CUtensorMap dmap{};
    const cudaError_t me = encode_disp_map(&dmap, disp, dp, g.W, g.H, IN, kGBW, kGBH);
    if (me != cudaSuccess) return me;
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_gate<IN, QMAP>, kGSmem, done);
    if (e != cudaSuccess) return e;
    const int ntiles = ((g.W + kTW - 1) / kTW) * ((g.H + kTH - 1) / kTH);
    const int grid = ntiles < 2 * sm_count() ? ntiles : 2 * sm_count();  // two resident CTAs per SM
    k_gate<IN, QMAP><<<grid, dim3(kTW, kTH), kGSmem, s>>>(g, o, gv, q, qp, dmap);
    return cudaGetLastError();
}

template <int IN>
cudaError_t launch_chain(const Geo& g, const void* disp, size_t dp, const FrameOut& o, cudaStream_t s) {
    CUtensorMap dmap{};
    const cudaError_t me = encode_disp_map(&dmap, disp, dp, g.W, g.H, IN, tma_bw<IN, kLR, kLTWR>(), kLTHR);
    if (me != cudaSuccess) return me;
    static std::atomic<unsigned long long> done{0};
    const cudaError_t e = smem_limit_once(k_learned<IN>, kCSmem, done);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.W + kTW - 1) / kTW, (g.H + kTH - 1) / kTH), block(kTW, kCThreads / kTW);
    k_learned<IN><<<grid, block, kCSmem, s>>>(g, static_cast<const char*>(disp), dp, o, dmap);
    return cudaGetLastError();
}

template <int IN>
cudaError_t launch_both(const Geo& g, const void* disp, size_t dp, const FrameOut& o, const GateView& gv, float* q,
                        size_t qp, cudaStream_t s) {
    if (q) return launch_gate<IN, true>(g, disp, dp, o, gv, q, qp, s);
    const cudaError_t e = launch_gate<IN, false>(g, disp, dp, o, gv, nullptr, 0, s);
    if (e != cudaSuccess) return e;
    return launch_chain<IN>(g, disp, dp, o, s);
}

std::mutex g_tab_mu;
bool g_tab_ready[64];

}  // namespace

cudaError_t log2_table(const float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_tab_mu);
    if (!g_tab_ready[dev]) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        k_log2tab<<<(kDMax + 1 + 255) / 256, 256, 0, st>>>();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (e != cudaSuccess) return e;
        g_tab_ready[dev] = true;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_log2tab);
    *out = static_cast<const float*>(p);
    return e;
}

}  // namespace sn

extern "C" sn_status sn_gate_log2_table(float* out, int n) {
    if (!out || n < sn::kDMax + 1) return SN_EINVAL;
    const float* t = nullptr;
    if (sn::log2_table(&t) != cudaSuccess) return SN_ECUDA;
    return cudaMemcpy(out, t, sizeof(float) * (sn::kDMax + 1), cudaMemcpyDeviceToHost) == cudaSuccess ? SN_OK
                                                                                                    : SN_ECUDA;
}

namespace sn {

cudaError_t launch_net_image(const GateView& gv, void* img, cudaStream_t s) {
    k_net_image<<<(16 * 144 + 255) / 256, 256, 0, s>>>(gv, static_cast<unsigned char*>(img));
    return cudaGetLastError();
}

cudaError_t launch_learned(const Geo& g, const void* disp, size_t dp, const FrameOut& o, const GateView& gv, float* q,
                           size_t qp, cudaStream_t s) {
    switch (g.in_dtype) {
        case SN_IN_F32: return launch_both<SN_IN_F32>(g, disp, dp, o, gv, q, qp, s);
        case SN_IN_F16: return launch_both<SN_IN_F16>(g, disp, dp, o, gv, q, qp, s);
        default: return launch_both<SN_IN_U16X256>(g, disp, dp, o, gv, q, qp, s);
    }
}

}  // namespace sn
