// BF16 patch-network layer on the 5th-generation tensor cores (sm_103a).
//
//   C[m][n] = epilogue( sum_k A[m][k] * W[n][k] ),  fp32 accumulation in TMEM
//   epilogue: z = scale[n] * acc + shift[n]; ReLU (hidden layers);
//             + R[m][n] (skip, Sec. 4); stored as bf16 (hidden) or fp32 (last)
//
// A (activations, [M][K]) and W ([N][K]) are both K-major.  One CTA per SM
// runs a persistent loop over 128 x BN output tiles (m-major order so the BN
// tiles of one row block run back to back and share the A rows in L2):
//   warp 0      TMA producer: 128 x 64 A and BN x 64 W boxes, 128-byte
//               swizzle, into a ring of STAGES shared-memory stages
//   warp 1      allocates TMEM and issues tcgen05.mma (M=128, N=BN, K=16)
//               from one thread; tcgen05.commit frees stages / publishes tiles
//   warps 2..9  epilogue: warp w reads TMEM lanes 32 (w % 4) ..; the two
//               warps of a lane quarter take alternate 32-column chunks
//               (tcgen05.ld 32 lanes x 32 columns), scale/shift/ReLU; bf16
//               outputs go through a swizzled 32 x 32 shared-memory box to a
//               TMA store, and the skip input comes in the same way by a TMA
//               load, so no lane issues global loads or stores per element
// Two TMEM accumulators let the epilogue of one tile overlap the MMAs of
// the next.  Every mbarrier wait is bounded (~1 s of %globaltimer); on
// expiry the thread records an error code in the caller's error word (one
// per context, so simulations sharing a device do not see each other's
// expiries), stops issuing work, and the CTA still meets at the final
// barrier, frees TMEM and returns.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "internal.h"

namespace dnnmg {

namespace {

enum TcErr { kErrFull = 1, kErrEmpty = 2, kErrTmemFull = 3, kErrTmemEmpty = 4, kErrDrain = 5, kErrSkip = 6 };

constexpr int BM = 128;
constexpr int BK = 64;                 // 64 bf16 = 128 bytes = one swizzle row
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = 64 + kEpiThreads;
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
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

// Bounded wait for the phase with the given parity; false on expiry (the
// error code is recorded once).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int code, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && globaltimer() - t0 > kWaitNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// Shared -> global tiled copy (bulk-group completion); coordinates past the
// tensor's extent are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(src), "r"(c0), "r"(c1)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the source shared memory of every committed store has been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... of every committed store but the most recent one
__device__ __forceinline__ void bulk_wait_read_all_but_last() {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// every committed store is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the async proxy (TMA)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core-matrix groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= uint64_t((addr & 0x3FFFF) >> 4);        // start address
    d |= uint64_t(1) << 16;                       // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;               // stride byte offset
    d |= uint64_t(1) << 46;                       // descriptor version (sm_100 family)
    d |= uint64_t(2) << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D fp32, A and B bf16,
// both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive fp32 columns from TMEM into registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int ACC_COLS = BN <= 128 ? 128 : 256;      // TMEM columns per accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS;              // power of two >= 32
    // per epilogue warp 4 KB: bf16 output box + skip box (2 KB each), or
    // one 32 x 32 fp32 staging block
    static constexpr int EP_WARP_BYTES = 4096;
    static constexpr int EP_BYTES = kEpiWarps * EP_WARP_BYTES;
    static constexpr int BAR_BYTES = 256;   // (2 STAGES + 5) barriers, TMEM slot (16), kEpiWarps skip barriers
    static constexpr int STAGES_FIT = (227 * 1024 - 1024 - BAR_BYTES - EP_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
    static constexpr int SMEM = STAGES * STAGE_BYTES + EP_BYTES + BAR_BYTES + 1024;
    static_assert(STAGES >= 2 && SMEM <= 227 * 1024, "shared memory per CTA");
    static_assert((2 * STAGES + 5) * 8 + 16 + kEpiWarps * 8 <= BAR_BYTES, "barrier area");
};

template <int BN, bool OUT_BF16>
__global__ void __launch_bounds__(kThreads, 1) tc_layer_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmW,
    const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmR,
    const float* __restrict__ scale, const float* __restrict__ shift, void* __restrict__ Cout, int64_t ldc,
    const __nv_bfloat16* __restrict__ R, int64_t ldr, int M, int N, int K, int relu, int withhold_first_load,
    int* __restrict__ err) {
    using C = Cfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;            // 1024-aligned stage buffers
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t ep_base = base + C::STAGES * C::STAGE_BYTES;        // 1024-aligned, 4 KB per epilogue warp
    float* ep_stage = reinterpret_cast<float*>(gbase + C::STAGES * C::STAGE_BYTES);
    const uint32_t bars = ep_base + C::EP_BYTES;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (C::STAGES + s); };
    auto tfull_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + b); };
    auto tempty_bar = [&](int b) { return bars + 8u * (2 * C::STAGES + 2 + b); };
    const uint32_t done_bar = bars + 8u * (2 * C::STAGES + 4);
    volatile uint32_t* tmem_slot = reinterpret_cast<volatile uint32_t*>(
        gbase + C::STAGES * C::STAGE_BYTES + C::EP_BYTES + (2 * C::STAGES + 5) * 8);
    auto skip_bar = [&](int w) { return bars + 8u * (2 * C::STAGES + 5) + 16u + 8u * w; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), kEpiThreads);
        }
        mbar_init(done_bar, 1);
        for (int w = 0; w < kEpiWarps; ++w) mbar_init(skip_bar(w), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmW)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(const_cast<uint32_t*>(tmem_slot))),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;

    const int tiles_n = (N + BN - 1) / BN;
    const int tiles_m = (M + BM - 1) / BM;
    const int total = tiles_m * tiles_n;
    const int kblocks = K / BK;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
            for (int kb = 0; kb < kblocks; ++kb) {
                if (!mbar_wait(empty_bar(stage), phase ^ 1u, kErrEmpty, err)) {
                    ok = false;
                    break;
                }
                const uint32_t sa = base + stage * C::STAGE_BYTES;
                mbar_arrive_expect_tx(full_bar(stage), C::STAGE_BYTES);
                // failure-path test: the first stage is armed but never
                // filled, so every wait that depends on it runs out
                if (!(withhold_first_load && t == int(blockIdx.x) && kb == 0)) {
                    tma_load_2d(sa, &tmA, full_bar(stage), kb * BK, m0);
                    tma_load_2d(sa + C::A_BYTES, &tmW, full_bar(stage), kb * BK, n0);
                }
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        // drain: every issued copy must land before the CTA exits.  The last
        // fill of stage s completed (or will complete) the full-barrier phase
        // with parity `phase` if s was filled in the current lap (s < stage),
        // else parity phase ^ 1 (a never-filled stage passes at once).
        for (int s = 0; s < C::STAGES; ++s)
            mbar_wait(full_bar(s), s < stage ? phase : (phase ^ 1u), kErrDrain, err);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t idesc = mma_idesc(BN);
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        int it = 0;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
            const int buf = it & 1;
            const uint32_t use = uint32_t(it >> 1);
            if (!mbar_wait(tempty_bar(buf), (use & 1u) ^ 1u, kErrTmemEmpty, err)) break;
            fence_after();
            const uint32_t d = tmem_base + uint32_t(buf * C::ACC_COLS);
            for (int kb = 0; kb < kblocks; ++kb) {
                if (!mbar_wait(full_bar(stage), phase, kErrFull, err)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t sa = base + stage * C::STAGE_BYTES;
                const uint64_t da = smem_desc(sa), db = smem_desc(sa + C::A_BYTES);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)   // +32 bytes per K=16 step inside the swizzle row
                    mma_bf16(d, da + uint64_t(2 * k), db + uint64_t(2 * k), idesc, (kb | k) != 0);
                mma_commit(empty_bar(stage));
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            mma_commit(tfull_bar(buf));
        }
        // all MMAs this thread issued must finish before TMEM is freed
        mma_commit(done_bar);
        mbar_wait(done_bar, 0, kErrDrain, err);
    } else if (warp >= 2) {
        // ---------------- epilogue: warp w reads TMEM lanes 32 (w % 4) ..
        // (its 32 rows) and the 32-column chunks c0 = 32 half, 32 half + 64, ...
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int ew = warp - 2;
        float* stage = ep_stage + ew * (C::EP_WARP_BYTES / 4);          // fp32 output
        const uint32_t obox0 = ep_base + uint32_t(ew * C::EP_WARP_BYTES);  // bf16 output box
        const uint32_t rbox = obox0 + 2048u;                              // skip input box
        const uint32_t rbar = skip_bar(ew);
        const bool has_r = OUT_BF16 && R != nullptr;
        // without a skip input its box is a second output box: consecutive
        // chunks alternate between the two, so a chunk's box writes wait
        // only for the store before the previous one
        uint32_t n_stored = 0;
        uint32_t rphase = 0;
        bool r_pending = false;
        // TMA load of the skip box of chunk c0 of the tile at (m0, n0)
        auto issue_skip = [&](int m0, int n0, int c0) {
            if (lane == 0) {
                mbar_arrive_expect_tx(rbar, 2048u);
                tma_load_2d(rbox, &tmR, rbar, n0 + c0, m0 + quarter * 32);
            }
            r_pending = true;
        };
        int it = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++it) {
            const int buf = it & 1;
            const uint32_t use = uint32_t(it >> 1);
            const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
            const int64_t row0 = int64_t(m0) + quarter * 32;
            const bool rows_live = row0 < M;                 // warp-uniform
            if (has_r && rows_live && n0 + half * 32 < N) issue_skip(m0, n0, half * 32);   // in flight during the wait
            // the wait result is made warp-uniform (the TMEM loads below are
            // warp-collective); a warp whose wait expired leaves on its own,
            // and the others' waits for it are bounded too
            const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull_bar(buf), use & 1u, kErrTmemFull, err));
            if (!ok) break;
            fence_after();
#pragma unroll 1
            for (int c0 = half * 32; c0 < BN; c0 += 64) {
                float v[32];
                const uint32_t taddr = tmem_base + (uint32_t(quarter * 32) << 16) + uint32_t(buf * C::ACC_COLS + c0);
                tmem_ld32(taddr, v);
                const int n_base = n0 + c0;
                // warp-uniform: later chunks are past N too; rows past M have nothing to store
                if (n_base >= N || !rows_live) continue;
                // per-column scale / shift (the same address in every lane: L1 broadcast)
                if (n_base + 32 <= N) {
                    const float4* sc4 = reinterpret_cast<const float4*>(scale + n_base);
                    const float4* sh4 = reinterpret_cast<const float4*>(shift + n_base);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 a = __ldg(sc4 + j), b = __ldg(sh4 + j);
                        v[4 * j] = fmaf(a.x, v[4 * j], b.x);
                        v[4 * j + 1] = fmaf(a.y, v[4 * j + 1], b.y);
                        v[4 * j + 2] = fmaf(a.z, v[4 * j + 2], b.z);
                        v[4 * j + 3] = fmaf(a.w, v[4 * j + 3], b.w);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int n = n_base + i;
                        v[i] = n < N ? fmaf(__ldg(scale + n), v[i], __ldg(shift + n)) : 0.f;
                    }
                }
                if (relu) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
                }
                if constexpr (OUT_BF16) {
                    // A 32 x 32 bf16 box in shared memory, as the 64-byte TMA
                    // swizzle lays it out: row r (this lane) at r * 64, its
                    // 16-byte piece j at piece j ^ ((r >> 1) & 3); both the
                    // row writes and the row reads are bank-conflict-free.
                    const uint32_t row_off = uint32_t(lane) * 64u;
                    const uint32_t sw = uint32_t((lane >> 1) & 3);
                    if (has_r) {
                        if (!mbar_wait(rbar, rphase, kErrSkip, err)) { /* recorded; values are garbage */ }
                        rphase ^= 1u;
                        r_pending = false;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            uint4 r;
                            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                                         : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                                         : "r"(rbox + row_off + ((uint32_t(j) ^ sw) << 4)));
                            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&r);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 f = __bfloat1622float2(h[e]);
                                v[8 * j + 2 * e] += f.x;
                                v[8 * j + 2 * e + 1] += f.y;
                            }
                        }
                        __syncwarp();                      // every lane has read the skip box
                        if (c0 + 64 < BN && n_base + 64 < N) issue_skip(m0, n0, c0 + 64);
                    }
                    const uint32_t obox = has_r ? obox0 : obox0 + ((n_stored & 1u) << 11);
                    // the last store from this box must have read it
                    if (lane == 0) {
                        if (has_r)
                            bulk_wait_read();
                        else
                            bulk_wait_read_all_but_last();
                    }
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        uint32_t o[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const __nv_bfloat162 hb = __floats2bfloat162_rn(v[8 * j + 2 * e], v[8 * j + 2 * e + 1]);
                            o[e] = *reinterpret_cast<const uint32_t*>(&hb);
                        }
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                                     ::"r"(obox + row_off + ((uint32_t(j) ^ sw) << 4)), "r"(o[0]), "r"(o[1]),
                                       "r"(o[2]), "r"(o[3])
                                     : "memory");
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmC, obox, n_base, int(row0));
                        bulk_commit();
                    }
                    ++n_stored;
                } else {
                    // fp32 rows of arbitrary stride: through a 32 x 32 block in
                    // shared memory (row r's float4 number q at q ^ (r & 7),
                    // conflict-free both ways), then a warp writes 32
                    // consecutive columns of one row
                    float4* srow = reinterpret_cast<float4*>(stage + lane * 32);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        srow[j ^ (lane & 7)] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    __syncwarp();
                    const int n = n_base + lane;
                    const int q = lane >> 2, e = lane & 3;
                    for (int r = 0; r < 32; ++r) {
                        const int64_t rw = row0 + r;
                        if (rw < M && n < N)
                            static_cast<float*>(Cout)[rw * ldc + n] = stage[r * 32 + ((q ^ (r & 7)) << 2) + e];
                    }
                    __syncwarp();
                }
            }
            fence_before();
            mbar_arrive(tempty_bar(buf));
        }
        // drain: a skip load still in flight (only after an early exit) and
        // every output store must complete before the CTA exits
        if (r_pending) mbar_wait(rbar, rphase, kErrDrain, err);
        if constexpr (OUT_BF16) {
            if (lane == 0) bulk_wait_all();
        }
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

// ---- host side ---------------------------------------------------------------

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D bf16 tensor [rows][cols] with row stride ld (elements), box
// [box_rows][box_cols]: operand boxes are 64 columns (128 bytes, 128-byte
// swizzle), epilogue boxes 32 x 32 (64 bytes, 64-byte swizzle).
bool make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
              int box_cols = BK, CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
    cuuint64_t strides[1] = {cuuint64_t(ld * 2)};
    cuuint32_t box[2] = {cuuint32_t(box_cols), cuuint32_t(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int BN, bool OUT_BF16>
cudaError_t launch_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* W, int64_t ldw, int n_rows_w,
                      const float* scale, const float* shift, void* C, int64_t ldc, const __nv_bfloat16* R,
                      int64_t ldr, int64_t M, int N, int K, bool relu, cudaStream_t s, int withhold, int* err) {
    using Cf = Cfg<BN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_layer_kernel<BN, OUT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Cf::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap ta, tw, tc = {}, tr = {};
    if (!make_map(&ta, A, M, K, lda, BM) || !make_map(&tw, W, n_rows_w, K, ldw, BN)) return cudaErrorInvalidValue;
    // bf16 output and skip input as [M][N] tensors in 32 x 32 boxes (the
    // store clips at M and N)
    if (OUT_BF16 && !make_map(&tc, C, M, N, ldc, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B)) return cudaErrorInvalidValue;
    if (OUT_BF16 && R && !make_map(&tr, R, M, N, ldr, 32, 32, CU_TENSOR_MAP_SWIZZLE_64B)) return cudaErrorInvalidValue;
    const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int grid = int(std::min<int64_t>(tiles, sm_count()));
    tc_layer_kernel<BN, OUT_BF16><<<grid, kThreads, Cf::SMEM, s>>>(ta, tw, tc, tr, scale, shift, C, ldc, R, ldr, int(M),
                                                                    N, K, relu ? 1 : 0, withhold, err);
    return cudaGetLastError();
}

}  // namespace

// Hidden layer (bf16 out) or last layer (fp32 out) of the BF16 network.
// Requirements (checked): K % 64 == 0, lda/ldw multiples of 8, 16-byte
// aligned A and W, M < 2^31, err a device int.  n_rows_w = rows stored in W
// (>= N).
cudaError_t launch_layer_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* W, int64_t ldw, int n_rows_w,
                            const float* scale, const float* shift, void* C, int64_t ldc, bool out_bf16,
                            const __nv_bfloat16* R, int64_t ldr, int64_t M, int N, int K, bool relu,
                            cudaStream_t s, int* err, int withhold_first_load) {
    if (M <= 0) return cudaSuccess;
    if (!err) return cudaErrorInvalidValue;
    if (K % BK || lda % 8 || ldw % 8 || (reinterpret_cast<uintptr_t>(A) & 15) ||
        (reinterpret_cast<uintptr_t>(W) & 15) || M >= (int64_t(1) << 31) || n_rows_w < N)
        return cudaErrorInvalidValue;
    if (out_bf16 && (ldc % 8 || (reinterpret_cast<uintptr_t>(C) & 15) || (R && (ldr % 8 || (reinterpret_cast<uintptr_t>(R) & 15)))))
        return cudaErrorInvalidValue;
    if (N <= 96)
        return out_bf16 ? launch_tc<96, true>(A, lda, W, ldw, n_rows_w, scale, shift, C, ldc, R, ldr, M, N, K, relu, s,
                                              withhold_first_load, err)
                        : launch_tc<96, false>(A, lda, W, ldw, n_rows_w, scale, shift, C, ldc, R, ldr, M, N, K, relu, s,
                                               withhold_first_load, err);
    return out_bf16 ? launch_tc<256, true>(A, lda, W, ldw, n_rows_w, scale, shift, C, ldc, R, ldr, M, N, K, relu, s,
                                           withhold_first_load, err)
                    : launch_tc<256, false>(A, lda, W, ldw, n_rows_w, scale, shift, C, ldc, R, ldr, M, N, K, relu, s,
                                            withhold_first_load, err);
}

// Read and clear an error word of the tensor-core kernels, in order on
// stream s (synchronises s).
cudaError_t read_tc_error(int* err, cudaStream_t s, int* code) {
    *code = 0;
    if (!err) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(code, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*code) {
        e = cudaMemsetAsync(err, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e;
}

}  // namespace dnnmg
