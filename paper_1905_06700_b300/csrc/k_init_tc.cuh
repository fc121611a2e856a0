// k_init_tc.cuh -- per-pixel initialisation (Methods, "3D Reconstruction
// algorithm") with the log-matched filter as a Toeplitz contraction on the
// tensor cores: tcgen05.mma with FP16 or BF16 operands and FP32 accumulators
// in tensor memory, histogram blocks staged by TMA.
//
// Exactness.  The filter is y(tau) = sum_s z(tau + s - origin) K_s with
// integer counts z and integer taps K_s.  The histogram is never converted:
// its raw uint16 words are the A operand.  As FP16, a word z < 1024 is the
// subnormal z 2^-24 (exact); as BF16, a word z < 128 is the subnormal
// z 2^-133 and the taps are stored as K_s 2^100.  Every product is then an
// exact multiple of the unit 2^-24 (FP16) or 2^-33 (BF16), and so is every
// partial sum while the pixel's photons times max K stay below 2^24 (checked;
// a pixel outside either limit raises the range status).  The filter output
// is therefore the same integer as the CUDA-core path's, and comparisons on
// the raw FP32 bits (non-negative) order it exactly.
//
// Shapes.  A CTA owns 128 pixels (MMA M, tensor-memory lanes) and streams
// their histograms in 64-bin blocks (one 128-byte swizzle row per pixel).
// Output tile j (positions 64j .. 64j + 63) reads blocks j + dlo .. j + dhi;
// for each block offset d the B operand is the 128 x 64 band
//   rows  0..63 : B[n][i] = K_{64 d + i - n + origin}   (filter)
//   rows 64..127: B[n][i] = 1 where that tap exists      (IRF-window count)
// so one N = 128 MMA chain leaves y and the window photon count W side by
// side in 128 accumulator columns; 16-bin K-steps whose taps are all zero are
// skipped.
//
// Roles (one CTA per SM, persistent over 128-pixel tiles):
//   warp 4      TMA producer: block (pixel tile, b) -> stage ring;
//   warp 5      MMA issuer (one thread), owns the tensor memory;
//   warps 0..3  epilogue, one thread per pixel (its tensor-memory lane):
//     - compaction of each block into the pixel's nonzero-bin entries (the
//       sparse form the PALM loop iterates over), photon totals, limits;
//     - peak picking: a position is a candidate when it is an immediate local
//       maximum (strict left, non-strict right), holds at least min_photons
//       in its IRF window and beats the pixel's current K-th best; the full
//       +-sep test reads a two-tile ring of y in shared memory; candidates
//       near a tile end wait for the next tile;
//     - after the last tile: b0 and r0 from the entries, as the CUDA-core path.
// Every wait is bounded (KParams::wait_ns, one second by default); on expiry
// the CTA raises the timeout status, the other roles leave their loops, the
// copies and MMAs in flight are awaited (each drain bounded by kTcDrainNs)
// and the tensor memory is freed.
#pragma once
#include "rt3d_device.cuh"

namespace rt3d {

constexpr int kTcRows = 128;                      // pixels per tile
constexpr int kTcBlk = 64;                        // bins per block
constexpr int kTcN = 128;                         // MMA N: 64 outputs + 64 window counts
constexpr int kTcAccBufs = 4;                     // accumulators of 128 columns
constexpr int kTcTmemCols = kTcAccBufs * kTcN;    // 512
constexpr int kTcStageBytes = kTcRows * kTcBlk * 2;
constexpr int kTcBBytes = kTcN * kTcBlk * 2;
constexpr int kTcRingStride = 2 * kTcBlk + 4;     // ints per pixel row (padded: no bank conflicts)
constexpr int kTcRingBytes = kTcRows * kTcRingStride * 4;
constexpr int kTcMaxSep = 32;
constexpr int kTcMaxStages = 8;
constexpr int kTcEpiWarps = 4;
constexpr int kTcThreads = (kTcEpiWarps + 2) * 32;
constexpr int kTcBarBytes = 1024;
constexpr int kTcSmemLimit = 227 * 1024;
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // default bound of every wait (KParams::wait_ns)
constexpr unsigned long long kTcDrainNs = 1000000000ull;  // bound of the teardown drains (copies, MMAs)

__host__ __device__ constexpr int tc_smem_bytes(int nd, int stages)
{
    return 1024 /* alignment slack */ + (nd + stages) * kTcStageBytes + kTcRingBytes + kTcBarBytes;
}

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// As above, but the thread may sleep (up to about 1 ms) until the phase completes.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity.  Gives up once the
// CTA's abort flag is raised or after `limit` ns, raising the flag itself
// (limit 0: gives up unless the phase has already completed).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (*abort_flag) return false;
        if (global_ns() - t0 >= limit) {
            *abort_flag = 1;
            return false;
        }
        if (mbar_try_wait_sleep(bar, parity)) return true;
    }
}

// Wait for a phase regardless of the abort flag, bounded by kTcDrainNs: used
// at teardown for copies and MMAs still in flight (after an abort).
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait_sleep(bar, parity))
        if (global_ns() - t0 > kTcDrainNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x,
                                            int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     (unsigned long long)map)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 128-byte-swizzled K-major operand: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor: FP32 accumulator, A and B both FP16
// (bf16 = 0) or both BF16 (bf16 = 1), both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(int bf16)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(kTcN >> 3) << 17) |
           ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


// ------------------------------------------------------------------ kernel

// Candidate at tau (value yc, raw bits) passes the full +-sep test: strictly
// above the sep positions before it, not below the sep positions after it
// (positions outside [0, T) do not count; q = 1 was tested already).
__device__ __forceinline__ bool tc_window_ok(const int* rrow, int tau, int yc, int sep, int T)
{
    const int lo = tau - min(sep, tau), hi = tau + min(sep, T - 1 - tau);
    // aligned 4-position groups covering [lo, hi]; the ring length (128) is a
    // multiple of 4, so a group never wraps
    bool bad = false;
    for (int p4 = lo & ~3; p4 <= hi; p4 += 4) {
        const int4 v = *reinterpret_cast<const int4*>(rrow + (p4 & 127));
        const int e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = p4 + k;
            bad |= (p >= lo) & (p < tau - 1) & (e[k] >= yc);
            bad |= (p > tau + 1) & (p <= hi) & (e[k] > yc);
        }
    }
    return !bad;
}

// Insert (y, tau) into the pixel's list ordered by y descending; candidates
// arrive in increasing tau, so an equal y keeps the earlier bin first.
__device__ __forceinline__ void tc_insert(int (&by)[kMaxK], int (&bt)[kMaxK], int& nb, int K, int y,
                                          int tau)
{
    int pos = nb;
#pragma unroll
    for (int k = kMaxK - 1; k >= 0; --k)
        if (k < nb && by[k] < y) pos = k;
    if (pos >= K) return;
#pragma unroll
    for (int k = kMaxK - 1; k > 0; --k)
        if (k > pos && k < K) {
            by[k] = by[k - 1];
            bt[k] = bt[k - 1];
        }
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
        if (k == pos) {
            by[k] = y;
            bt[k] = tau;
        }
    if (nb < K) ++nb;
}

template <bool kDumpY>
__global__ void __launch_bounds__(kTcThreads, 1)
k_init_tc(const CallRecord* __restrict__ rec, const Work W, const uint8_t* __restrict__ bimg, int tc0, int tc1)
{
    const KParams& P = rec->P;
    const Batch& B = rec->B;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    const int nd = P.tc_nd, S = P.tc_stages, dlo = P.tc_dlo;
    const uint32_t sB = base;                                   // nd band operands
    const uint32_t sA = base + (uint32_t)nd * kTcBBytes;        // S histogram stages
    int* ring = reinterpret_cast<int*>(gbase + (size_t)(nd + S) * kTcStageBytes);
    unsigned char* misc_g = gbase + (size_t)(nd + S) * kTcStageBytes + kTcRingBytes;
    const uint32_t misc = base + (uint32_t)(nd + S) * kTcStageBytes + kTcRingBytes;
    // barriers: full[S], empty[S], acc_full[4], acc_empty[4]; then tmem base,
    // abort flag, the MMA drain barrier
    const uint32_t bar_full = misc, bar_empty = misc + 8 * kTcMaxStages;
    const uint32_t bar_accf = misc + 16 * kTcMaxStages, bar_acce = bar_accf + 8 * kTcAccBufs;
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(misc_g + 16 * kTcMaxStages + 16 * kTcAccBufs);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(misc_g + 16 * kTcMaxStages + 16 * kTcAccBufs + 4);
    const uint32_t bar_drain = misc + 16 * kTcMaxStages + 16 * kTcAccBufs + 8;
    const unsigned long long wlim = P.wait_ns;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // band operands -> shared memory (generic writes, then visible to the tensor cores)
    {
        const uint4* src = reinterpret_cast<const uint4*>(bimg);
        uint4* dst = reinterpret_cast<uint4*>(gbase);
        const int n16 = nd * kTcBBytes / 16;
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1 + kTcEpiWarps);
        }
        for (int a = 0; a < kTcAccBufs; ++a) {
            mbar_init(bar_accf + 8 * a, 1);
            mbar_init(bar_acce + 8 * a, kTcEpiWarps);
        }
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcEpiWarps + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32((const void*)tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kTcEpiWarps) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t g = 0;
            bool stop = false;
            for (int tile = tc0 + (int)blockIdx.x; tile < tc1 && !stop; tile += gridDim.x) {
                const int f = frame_of_tc_tile(B, tile);
                const FrameDesc& F = B.f[f];
                const int pt = tile - F.tc_tile_base;
                const int nbk = (F.nt + kTcBlk - 1) / kTcBlk;
                const CUtensorMap* map = &rec->maps[f];
                tmap_acquire(map);
                for (int b = 0; b < nbk; ++b, ++g) {
                    const uint32_t s = g % (uint32_t)S;
                    if (g >= (uint32_t)S && !mbar_wait(bar_empty + 8 * s, ((g / S) & 1u) ^ 1u, abort_flag, wlim)) {
                        stop = true;
                        break;
                    }
                    mbar_expect_tx(bar_full + 8 * s, kTcStageBytes);
                    tma_load_2d(sA + s * kTcStageBytes, map, bar_full + 8 * s, b * kTcBlk, pt * kTcRows);
                }
            }
            // copies in flight land before the CTA may exit: the last load of
            // each stage completes its full barrier
            for (uint32_t k = 0; k < (uint32_t)S && k < g; ++k) {
                const uint32_t last = g - 1 - k;
                mbar_drain(bar_full + 8 * (last % (uint32_t)S), (last / S) & 1u);
            }
        }
    } else if (warp == kTcEpiWarps + 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(P.tc_mode == 1 ? 1 : 0);
            int ksmask[kTcMaxOff];            // kept in registers: read once
#pragma unroll
            for (int di = 0; di < kTcMaxOff; ++di) ksmask[di] = P.tc_ksmask[di];
            uint32_t g0 = 0, acc_cnt = 0;
            bool stop = false, issued = false;
            for (int tile = tc0 + (int)blockIdx.x; tile < tc1 && !stop; tile += gridDim.x) {
                const FrameDesc& F = B.f[frame_of_tc_tile(B, tile)];
                const int nbk = (F.nt + kTcBlk - 1) / kTcBlk;
                int rel = 0;   // next block whose stage is still held by the MMA
                for (int j = 0; j < nbk && !stop; ++j, ++acc_cnt) {
                    const uint32_t a = acc_cnt % kTcAccBufs;
                    if (acc_cnt >= (uint32_t)kTcAccBufs &&
                        !mbar_wait(bar_acce + 8 * a, ((acc_cnt / kTcAccBufs) & 1u) ^ 1u, abort_flag, wlim)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + a * kTcN;
                    uint32_t accumulate = 0;
#pragma unroll
                    for (int di = 0; di < kTcMaxOff; ++di) {
                        if (di >= nd || stop) continue;
                        const int b = j + dlo + di;
                        if (b < 0 || b >= nbk) continue;
                        const uint32_t gb = g0 + (uint32_t)b;
                        const uint32_t s = gb % (uint32_t)S;
                        // TMA completion is observed through the barrier; the MMA
                        // reads the stage in the same (async) proxy
                        if (!mbar_wait(bar_full + 8 * s, (gb / S) & 1u, abort_flag, wlim)) {
                            stop = true;
                            break;
                        }
                        const int mask = ksmask[di];
                        for (int ks = 0; ks < 4; ++ks) {
                            // the block of offset 0 always issues its first step, so
                            // every accumulator is written even for an all-zero band
                            if (!((mask >> ks) & 1) && !(b == j && ks == 0 && !accumulate)) continue;
                            tc_mma(dt, tc_desc_sw128(sA + s * kTcStageBytes + ks * 32),
                                   tc_desc_sw128(sB + di * kTcBBytes + ks * 32), idesc, accumulate);
                            accumulate = 1;
                            issued = true;
                        }
                    }
                    if (stop) break;
                    tc_commit(bar_accf + 8 * a);
                    // stages whose last reader was this tile
                    const int hi = (j == nbk - 1) ? nbk - 1 : j + dlo;
                    for (; rel <= hi; ++rel) tc_commit(bar_empty + 8 * ((g0 + (uint32_t)rel) % (uint32_t)S));
                }
                g0 += (uint32_t)nbk;
            }
            // every MMA has finished before the tensor memory is freed (after an
            // abort some were issued without a commit the epilogue waited for)
            if (issued) {
                tc_commit(bar_drain);
                mbar_drain(bar_drain, 0u);
            }
        }
    } else {
        // ------------------------------------------------ epilogue: one pixel per thread
        const int row = warp * 32 + lane;
        const int K = P.k, O = P.irf_origin, L = P.irf_len, sep = P.peak_sep;
        const int dhi = dlo + nd - 1;
        const int wmin = P.tc_wmin_bits;
        int* rrow = ring + row * kTcRingStride;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        uint32_t g0 = 0, acc_cnt = 0;
        bool stop = false;
        for (int tile = tc0 + (int)blockIdx.x; tile < tc1 && !stop; tile += gridDim.x) {
            const FrameDesc& F = B.f[frame_of_tc_tile(B, tile)];
            const int pt = tile - F.tc_tile_base;
            const int T = F.nt;
            const int nbk = (T + kTcBlk - 1) / kTcBlk;
            const int lp = pt * kTcRows + row;
            const bool valid = lp < F.npix;
            uint32_t* eout = const_cast<uint32_t*>(F.ent) + (long long)lp * T;
            uint32_t nnz = 0, zmax = 0;
            unsigned long long total = 0;
            int by[kMaxK], bt[kMaxK], nb = 0;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                by[k] = 0;
                bt[k] = 0;
            }
            int cy62 = -1, cy63 = -1;          // y at 64j - 2, 64j - 1 (raw bits; -1 = outside)
            bool cw63 = false;                  // window count test at 64j - 1
            uint64_t defer = 0;                 // candidates of the previous tile awaiting their right window
            int c_next = 0;                     // next block to compact

            for (int j = 0; j < nbk; ++j, ++acc_cnt) {
                const uint32_t a = acc_cnt % kTcAccBufs;
                // lanes agree on every wait's outcome (warp-collective steps follow)
                if (!__all_sync(0xffffffffu,
                                mbar_wait(bar_accf + 8 * a, (acc_cnt / kTcAccBufs) & 1u, abort_flag, wlim))) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                uint32_t yv[64], wv[64];
                tc_ld32(lane_base + a * kTcN, *reinterpret_cast<uint32_t(*)[32]>(&yv[0]));
                tc_ld32(lane_base + a * kTcN + 32, *reinterpret_cast<uint32_t(*)[32]>(&yv[32]));
                tc_ld32(lane_base + a * kTcN + 64, *reinterpret_cast<uint32_t(*)[32]>(&wv[0]));
                tc_ld32(lane_base + a * kTcN + 96, *reinterpret_cast<uint32_t(*)[32]>(&wv[32]));
                tc_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acce + 8 * a);

                // positions past the histogram end do not exist
                const int tau0 = j * kTcBlk;
                if (tau0 + kTcBlk > T) {
#pragma unroll
                    for (int i = 0; i < 64; ++i)
                        if (tau0 + i >= T) yv[i] = 0xffffffffu;
                }

                // compaction of the blocks this tile's window reaches
                const int chi = min(j + dhi, nbk - 1);
                for (; c_next <= chi; ++c_next) {
                    const uint32_t gb = g0 + (uint32_t)c_next;
                    const uint32_t s = gb % (uint32_t)S;
                    if (!__all_sync(0xffffffffu, mbar_wait(bar_full + 8 * s, (gb / S) & 1u, abort_flag, wlim))) {
                        stop = true;
                        break;
                    }
                    const unsigned char* srow = gbase + (size_t)(nd + s) * kTcStageBytes + row * 128;
                    // 16-byte chunk c (bins 8c .. 8c + 7) sits at chunk c ^ (row & 7)
                    uint32_t nzc = 0;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const uint4 q = *reinterpret_cast<const uint4*>(srow + ((c ^ (row & 7)) << 4));
                        nzc |= (uint32_t)((q.x | q.y | q.z | q.w) != 0u) << c;
                    }
                    if (valid) {
                        // a lane's loop runs over its own nonzero chunks only
                        const uint32_t bin0 = (uint32_t)c_next * kTcBlk;
                        while (nzc) {
                            const int c = __ffs(nzc) - 1;
                            nzc &= nzc - 1;
                            const uint4 q = *reinterpret_cast<const uint4*>(srow + ((c ^ (row & 7)) << 4));
                            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                            for (int h = 0; h < 8; ++h) {
                                const uint32_t z = (w4[h >> 1] >> ((h & 1) * 16)) & 0xffffu;
                                if (!kDumpY && z) eout[nnz++] = ((bin0 + 8 * c + h) << 16) | z;
                                total += z;
                                zmax = max(zmax, z);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar_empty + 8 * s);
                }
                if (stop) break;

                if constexpr (kDumpY) {
                    if (valid) {
                        int* yo = W.y_out + (long long)lp * T + tau0;
#pragma unroll
                        for (int i = 0; i < 64; ++i)
                            if (tau0 + i < T) yo[i] = __float2int_rn(__uint_as_float(yv[i]) * P.tc_unit_inv);
                    }
                    continue;
                } else {
                    // this tile's y into the ring
                    {
                        int4* dst = reinterpret_cast<int4*>(rrow + (j & 1) * 64);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            dst[i] = make_int4((int)yv[4 * i], (int)yv[4 * i + 1], (int)yv[4 * i + 2],
                                               (int)yv[4 * i + 3]);
                    }
                    int thr = nb == K ? by[K - 1] : 0;
                    // previous tile's last position (its right neighbour is here)
                    if (j > 0 && cy63 > max(thr, cy62) && cy63 >= (int)yv[0] && cw63)
                        defer |= 1ull << 63;
                    // previous tile's deferred candidates, in increasing position
                    while (defer) {
                        const int i = __ffsll((long long)defer) - 1;
                        defer &= defer - 1;
                        const int tau = tau0 - 64 + i;
                        const int yc = rrow[tau & 127];
                        const int th = nb == K ? by[K - 1] : 0;
                        if (yc > th && tc_window_ok(rrow, tau, yc, sep, T)) tc_insert(by, bt, nb, K, yc, tau);
                    }
                    thr = nb == K ? by[K - 1] : 0;
                    // immediate local maxima of this tile (positions 0 .. 62)
                    // eight independent 8-bit accumulators keep the dependency chains short
                    uint32_t cb[8];
#pragma unroll
                    for (int g8 = 0; g8 < 8; ++g8) {
                        uint32_t m = 0;
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int i = 8 * g8 + k;
                            if (i < 63) {
                                const int yl = i == 0 ? cy63 : (int)yv[i - 1];
                                const int yi = (int)yv[i];
                                const bool c = (yi > max(thr, yl)) & (yi >= (int)yv[i + 1]) & ((int)wv[i] >= wmin);
                                m |= (uint32_t)c << k;
                            }
                        }
                        cb[g8] = m;
                    }
                    const uint32_t clo = cb[0] | (cb[1] << 8) | (cb[2] << 16) | (cb[3] << 24);
                    const uint32_t chi2 = cb[4] | (cb[5] << 8) | (cb[6] << 16) | (cb[7] << 24);
                    const uint64_t cand = ((uint64_t)chi2 << 32) | clo;
                    cy62 = (int)yv[62];
                    cy63 = (int)yv[63];
                    cw63 = (int)wv[63] >= wmin;
                    // candidates whose right window ends inside this tile now, the rest later
                    const uint64_t now_mask = (sep >= 63) ? 0ull : ((1ull << (64 - sep)) - 1ull);
                    uint64_t now = cand & now_mask;
                    defer = cand & ~now_mask;
                    while (now) {
                        const int i = __ffsll((long long)now) - 1;
                        now &= now - 1;
                        const int tau = tau0 + i;
                        const int yc = rrow[tau & 127];
                        const int th = nb == K ? by[K - 1] : 0;
                        if (yc > th && tc_window_ok(rrow, tau, yc, sep, T)) tc_insert(by, bt, nb, K, yc, tau);
                    }
                }
            }
            if (stop) break;
            g0 += (uint32_t)nbk;
            if (kDumpY || !valid) continue;

            // the histogram's last position (no right neighbour) and the last deferred candidates
            {
                const int i_last = (T - 1) & 63;
                const int th = nb == K ? by[K - 1] : 0;
                if (i_last == 63 && cy63 > th && cy63 > cy62 && cw63) defer |= 1ull << 63;
                const int tau0 = (nbk - 1) * kTcBlk;
                while (defer) {
                    const int i = __ffsll((long long)defer) - 1;
                    defer &= defer - 1;
                    const int tau = tau0 + i;
                    const int yc = rrow[tau & 127];
                    const int t2 = nb == K ? by[K - 1] : 0;
                    if (yc > t2 && tc_window_ok(rrow, tau, yc, sep, T)) tc_insert(by, bt, nb, K, yc, tau);
                }
            }

            // ---- initial intensities and background (as the CUDA-core path)
            const float g = F.gain ? F.gain[lp] : 1.0f;
            const bool in_range = total * (unsigned long long)P.lmf_kmax < (1ull << 24) &&
                                  zmax < (uint32_t)P.tc_count_limit;
            if (!in_range) atomicOr(W.status, kStatusRange);
            int nsel = (in_range && g > 0.0f) ? nb : 0;
            int sel[kMaxK];
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) sel[k] = bt[k];
            // slots by increasing depth
#pragma unroll
            for (int a2 = 0; a2 < kMaxK; ++a2)
#pragma unroll
                for (int c2 = a2 + 1; c2 < kMaxK; ++c2)
                    if (c2 < nb && sel[c2] < sel[a2]) {
                        const int tmp = sel[a2];
                        sel[a2] = sel[c2];
                        sel[c2] = tmp;
                    }
            unsigned long long inside = 0;
            unsigned long long wsum[kMaxK] = {0, 0, 0, 0};
            for (uint32_t e = 0; e < nnz; ++e) {
                const uint32_t v = eout[e];
                const int bin = (int)(v >> 16);
                const unsigned z = v & 0xffffu;
                bool any = false;
#pragma unroll
                for (int k = 0; k < kMaxK; ++k)
                    if (k < nb && bin >= sel[k] - O && bin <= sel[k] - O + L - 1) {
                        wsum[k] += z;
                        any = true;
                    }
                if (any) inside += z;
            }
            int covered = 0, cur_lo = 0, cur_hi = -1;
            int winlen[kMaxK];
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                winlen[k] = 0;
                if (k >= nb) continue;
                const int lo = max(sel[k] - O, 0), hi = min(sel[k] - O + L - 1, T - 1);
                winlen[k] = max(hi - lo + 1, 0);
                if (hi < lo) continue;
                if (lo > cur_hi) {
                    covered += max(cur_hi - cur_lo + 1, 0);
                    cur_lo = lo;
                    cur_hi = hi;
                } else if (hi > cur_hi) {
                    cur_hi = hi;
                }
            }
            covered += max(cur_hi - cur_lo + 1, 0);
            const long long t_out = (long long)T - covered;
            const long long n_out = (long long)total - (long long)inside;
            float b0 = P.b_floor;
            if (g > 0.0f && t_out > 0) b0 = fmaxf((float)n_out / ((float)t_out * g), P.b_floor);
            const int np = F.npix;
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) {
                if (k >= K) continue;
                const bool on = k < nsel;
                F.t[(long long)k * np + lp] = on ? (float)sel[k] : 0.0f;
                F.r[(long long)k * np + lp] = on ? fmaxf((float)wsum[k] / g - b0 * (float)winlen[k], P.r_min) : 0.0f;
                F.alive[(long long)k * np + lp] = on ? 1 : 0;
            }
            F.b[lp] = b0;
            W.seg[F.pix_base + lp] = make_uint2((uint32_t)((long long)lp * T), nnz);
            if (lp == 0 && F.n_points) *F.n_points = 0;
        }
    }

    // ---- teardown: every role has left its loop (all waits are bounded)
    if (*abort_flag && threadIdx.x == 0) atomicOr(W.status, kStatusTimeout);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kTcEpiWarps + 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols)
                     : "memory");
}

}  // namespace rt3d
