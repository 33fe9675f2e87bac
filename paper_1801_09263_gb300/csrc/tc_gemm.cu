// Tensor-core (tcgen05, sm_103a) split-precision contraction over the grid:
//   work[chunk][m][n] = sum_{r in chunk} op(A[m][r]) * op(B[n][r])
// for the dense ACE contractions (Eq. 3: M = dV Psi^T W; K_ACE psi needs
// X = dV xi^T psi) and the overlap of moduli (Eq. 4, op = |.|, A = B).  Each
// FP32 operand is split in registers into BF16 hi = bf16(x), lo = bf16(x - hi);
// the products hi.hi + hi.lo + lo.hi are accumulated in FP32 in tensor memory
// (the lo.lo term, ~2^-16 relative and of random sign between different
// operands, is dropped; the overlap of moduli keeps it).  Chunks of K are
// reduced in FP64 by the caller in a fixed order.
//
// Kernels:
// * tc_gram_ws_kernel (the Gram, default): one 128 x 128 output tile and one
//   K chunk per CTA (for A = B only the tiles on and above the diagonal); the
//   FP32 rows arrive by TMA (cp.async.bulk.tensor) four 32-wide steps ahead,
//   16 warps split them into BF16 hi/lo tiles (64-byte swizzled K-major, two
//   stages), one thread issues the tcgen05.mma (M128 N128 K16) and one the
//   copies; the roles hand off through mbarriers.  The MMAs accumulate a few
//   steps per TMEM accumulator (two alternating), which the split warps drain
//   into compensated FP32 sums.
// * tc_combine_tma_kernel (the combination, default): persistent over output
//   tiles of 128 grid points x 256 targets; the FP32 A tiles and the pre-split
//   coefficient tiles arrive by TMA (the latter directly in the 128-byte
//   swizzled layout), the threads transpose-split A; FP32 or FP64 output.
// * tc_gram_kernel / tc_combine_kernel: the same contractions with the
//   operands loaded through registers (used when no tensor map can be made).
// Every mbarrier wait is bounded; on a timeout the CTA records an error,
// drains what it started and returns.
#include <atomic>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lace_internal.cuh"

namespace lace {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_BK = 64, TC_THREADS = 512;
constexpr int TC_VPT = (TC_M * TC_BK / 4) / TC_THREADS;  // float4 vectors per thread per tile
constexpr int TC_TILE_BYTES = TC_M * TC_BK * 2;      // 16 KB per BF16 tile
constexpr int TC_STAGE_BYTES = 4 * TC_TILE_BYTES;    // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM_BYTES = 2 * TC_STAGE_BYTES + 1024;  // + alignment slack
constexpr long long TC_WAIT_LIMIT = 1LL << 26;       // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 128-byte swizzled K-major shared-memory descriptor (SBO = 1024 B between
// 8-row groups, version 1, layout type 2 = SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // SWIZZLE_128B
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                            ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Byte offset of BF16 element (row r, k) in a 128-byte swizzled K-major tile of 64 columns.
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

// Two FP32 values rounded to BF16 (round to nearest even) and packed: x0 in
// the low half (the lower address), x1 in the high half.
__device__ __forceinline__ uint32_t bf16x2_rn(float x0, float x1) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
    return r;
}

// hi = bf16(x), lo = bf16(x - hi) for four values, packed in element order
// (one conversion instruction per two values; a BF16 value widens to FP32
// exactly by placing its bits in the upper half).
__device__ __forceinline__ void split4(float4 v, uint2& hi, uint2& lo) {
    hi.x = bf16x2_rn(v.x, v.y);
    hi.y = bf16x2_rn(v.z, v.w);
    const float r0 = v.x - __uint_as_float(hi.x << 16), r1 = v.y - __uint_as_float(hi.x & 0xffff0000u);
    const float r2 = v.z - __uint_as_float(hi.y << 16), r3 = v.w - __uint_as_float(hi.y & 0xffff0000u);
    lo.x = bf16x2_rn(r0, r1);
    lo.y = bf16x2_rn(r2, r3);
}

// Load this thread's share of a 128 x 64 FP32 tile (rows row0.., columns
// k0..) into registers.  Rows >= nrows and columns >= kend read as zero.
__device__ __forceinline__ void load_tile(const float* __restrict__ src, size_t ld, int row0, int nrows, size_t k0,
                                          size_t kend, float4* v) {
#pragma unroll
    for (int j = 0; j < TC_VPT; ++j) {
        const int e = threadIdx.x + j * TC_THREADS;
        const int r = e >> 4, kv = (e & 15) * 4;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        const int row = row0 + r;
        const size_t k = k0 + kv;
        if (row < nrows && k < kend) {
            const float* p = src + (size_t)row * ld + k;
            if (k + 4 <= kend) {
                x = __ldg(reinterpret_cast<const float4*>(p));
            } else {
                x.x = p[0];
                if (k + 1 < kend) x.y = p[1];
                if (k + 2 < kend) x.z = p[2];
            }
        }
        v[j] = x;
    }
}

// Split the registers (or their absolute values) into BF16 hi/lo and store
// them in the swizzled tiles.
template <bool ABS>
__device__ __forceinline__ void store_tile(const float4* v, unsigned char* hi_tile, unsigned char* lo_tile) {
#pragma unroll
    for (int j = 0; j < TC_VPT; ++j) {
        const int e = threadIdx.x + j * TC_THREADS;
        const int r = e >> 4, kv = (e & 15) * 4;
        uint2 h, l;
        const float4 x = ABS ? make_float4(fabsf(v[j].x), fabsf(v[j].y), fabsf(v[j].z), fabsf(v[j].w)) : v[j];
        split4(x, h, l);
        const uint32_t off = sw128_off(r, kv);
        *reinterpret_cast<uint2*>(hi_tile + off) = h;
        *reinterpret_cast<uint2*>(lo_tile + off) = l;
    }
}

template <bool ABS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gram_kernel(int M, int N, size_t K, const float* __restrict__ A, size_t lda, const float* __restrict__ B,
                   size_t ldb, size_t kchunk, double* __restrict__ work, int* __restrict__ err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * TC_N;
    const size_t k_begin = (size_t)blockIdx.z * kchunk;
    const size_t k_end = min(K, k_begin + kchunk);
    const int nsteps = (int)((k_end - k_begin + TC_BK - 1) / TC_BK);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // 128 TMEM columns x 128 lanes of FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    uint32_t uses[2] = {0u, 0u};
    // one step of register prefetch: the rows of step t+1 are in flight while
    // step t is split, stored and handed to the tensor cores
    float4 va[TC_VPT], vb[TC_VPT];
    if (nsteps > 0) {
        load_tile(A, lda, m0, M, k_begin, k_end, va);
        load_tile(B, ldb, n0, N, k_begin, k_end, vb);
    }
    for (int step = 0; step < nsteps; ++step) {
        const int s = step & 1;
        unsigned char* st = smem + s * TC_STAGE_BYTES;
        if (uses[s] > 0) {
            // the MMAs that read this stage two steps ago must be done
            if (threadIdx.x == 0 && !mbar_wait(&bars[s], (uses[s] - 1) & 1)) abort_sh = 1;
            __syncthreads();
            if (abort_sh) break;
        }
        store_tile<ABS>(va, st, st + TC_TILE_BYTES);
        store_tile<ABS>(vb, st + 2 * TC_TILE_BYTES, st + 3 * TC_TILE_BYTES);
        if (step + 1 < nsteps) {
            const size_t k1 = k_begin + (size_t)(step + 1) * TC_BK;
            load_tile(A, lda, m0, M, k1, k_end, va);
            load_tile(B, ldb, n0, N, k1, k_end, vb);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(st), a_lo = a_hi + TC_TILE_BYTES;
            const uint32_t b_hi = a_hi + 2 * TC_TILE_BYTES, b_lo = a_hi + 3 * TC_TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint32_t ko = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzle atom
                const uint32_t first = (step == 0 && kk == 0) ? 0u : 1u;
                mma_bf16(tmem, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), first);
                mma_bf16(tmem, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), 1u);
                mma_bf16(tmem, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), 1u);
            }
            mma_commit(&bars[s]);
        }
        uses[s] += 1;
    }
    // wait for the last MMAs (commits complete in issue order)
    if (nsteps > 0 && !abort_sh) {
        const int s = (nsteps - 1) & 1;
        if (threadIdx.x == 0 && !mbar_wait(&bars[s], (uses[s] - 1) & 1)) abort_sh = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_sh) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else if (warp < 4 && nsteps > 0) {
        // warp w reads TMEM lanes 32w..32w+31 = output rows m0 + 32w + lane
        const int row = m0 + warp * 32 + (threadIdx.x & 31);
        double* out = work + (size_t)blockIdx.z * M * N;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N) out[(size_t)row * N + col] = (double)__uint_as_float(v[j]);
                }
            }
        }
    } else if (nsteps == 0 && warp < 4) {
        const int row = m0 + warp * 32 + (threadIdx.x & 31);
        double* out = work + (size_t)blockIdx.z * M * N;
        if (row < M)
            for (int j = 0; j < TC_N; ++j)
                if (n0 + j < N) out[(size_t)row * N + n0 + j] = 0.0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    }
}

// ---------------------------------------------------------------------------
// TMA helpers.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2D tile load: box at element coordinates (x = column, y = row) of the map.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Geometry of the TMA-fed Gram (tc_gram_ws_kernel): 32-wide K steps, so that
// two BF16 stages fit beside a deep FP32 pipeline: TG2_STAGES steps of 128 x
// 32 FP32 tiles of A and B in flight (plain row-major, 16 KB each), and two
// BF16 stages of the four split tiles (64-byte swizzled K-major, 8 KB each),
// so the split of step t overlaps the MMAs of step t - 1 and waits only for
// those of step t - 2.  An FP32 stage is refilled as soon as its step is split.
constexpr int TG2_BK = 32;
constexpr int TG2_STAGES = 4;
constexpr int TG2_F32_TILE = TC_M * TG2_BK * 4;       // 16 KB
constexpr int TG2_F32_STAGE = 2 * TG2_F32_TILE;       // A and B
constexpr int TG2_BF_TILE = TC_M * TG2_BK * 2;        // 8 KB
constexpr int TG2_BF_STAGE = 4 * TG2_BF_TILE;         // A_hi, A_lo, B_hi, B_lo
constexpr int TG2_SMEM_BYTES = TG2_STAGES * TG2_F32_STAGE + 2 * TG2_BF_STAGE + 1024;
constexpr int TG2_VPT = (TC_M * TG2_BK / 4) / TC_THREADS;  // float4 per thread per tile

// 64-byte swizzled K-major shared-memory descriptor (SBO = 512 B between
// 8-row groups, version 1, layout type 4 = SWIZZLE_64B).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Byte offset of BF16 element (row r, k) in a 64-byte swizzled K-major tile
// of 32 columns (16-byte chunk c of row r at chunk c ^ ((r / 2) mod 4)).
__device__ __forceinline__ uint32_t sw64_off(int r, int k) {
    return (uint32_t)(r * 64 + ((((k >> 3) ^ (r >> 1)) & 3) << 4) + (k & 7) * 2);
}

template <bool ABS>
__device__ __forceinline__ void split_tile32(const unsigned char* f32, unsigned char* hi_tile, unsigned char* lo_tile) {
#pragma unroll
    for (int j = 0; j < TG2_VPT; ++j) {
        const int e = threadIdx.x + j * TC_THREADS;
        const int r = e >> 3, kv = (e & 7) * 4;
        float4 v = *reinterpret_cast<const float4*>(f32 + (size_t)r * (TG2_BK * 4) + kv * 4);
        if (ABS) v = make_float4(fabsf(v.x), fabsf(v.y), fabsf(v.z), fabsf(v.w));
        uint2 h, l;
        split4(v, h, l);
        const uint32_t off = sw64_off(r, kv);
        *reinterpret_cast<uint2*>(hi_tile + off) = h;
        *reinterpret_cast<uint2*>(lo_tile + off) = l;
    }
}

// The 32-wide TMA-fed Gram with warp roles instead of CTA-wide barriers:
// warps 0-15 split (and drain the accumulators), warp 16 (lane 0) issues the
// TMA copies, warp 17 (lane 0) issues the MMAs.  They hand off through
// mbarriers only: full[s] (copies landed), empty[s] (stage s split, one
// arrival per splitting warp), split[b] (BF16 stage b written, one arrival
// per splitting warp) and mma[b] (the MMAs that read BF16 stage b are done;
// tcgen05.commit).  So the copies run TG2_STAGES steps ahead, the split of
// step t overlaps the MMAs of step t - 1, and no role waits for another
// except on data.  Every wait is bounded and also gives up once another role
// has recorded a timeout; the roles then drain what they started (bounded)
// and the CTA reports the error.
//
// Accumulation: the tensor cores add each K16 product block into the FP32
// accumulator with their own rounding, which over a K chunk of ~10^4 points
// biased the 256 x 256 ACE matrix of the 72^3 workload by -5.6e-6 relative
// (diagonal mean against FP64).  So the MMAs accumulate only TG2_DRAIN steps
// (128 products) into one of two TMEM accumulators; the split warps then read
// that period's sums (tcgen05.ld) and add them into compensated (Kahan) FP32
// registers, while the MMAs of the next period fill the other accumulator
// (measured bias: -2.1e-7 with 2-step periods, -6.1e-7 with 8-step periods).
// Split warp w owns TMEM lanes 32 (w mod 4).. (the lanes its warp may read)
// and columns 32 (w / 4)..
constexpr int TW_SPLIT_WARPS = 16;
constexpr int TW_THREADS = (TW_SPLIT_WARPS + 2) * 32;
constexpr int TG2_DRAIN = 4;  // steps per accumulation period
static_assert(TG2_DRAIN >= 2, "a period's drain follows the split of the next period's second step");

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when *abort is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    return false;
}

// 16 FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// Add one period's accumulator (32 columns at taddr) into the Kahan sums.
// The compensations are kept as BF16 pairs (comp2[j] holds columns 2j and
// 2j + 1): a compensation is below half an ulp of its sum, so its own 8-bit
// rounding costs ~2^-9 of that half ulp per period, and the 48 registers of
// state (instead of 64) leave room for the split.
__device__ __forceinline__ void drain_period(uint32_t taddr, float* fold, uint32_t* comp2) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[16];
        tmem_ld16(taddr + 16 * h, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const int q = 16 * h + j;
            const uint32_t c = comp2[q >> 1];
            const float y0 = __uint_as_float(v[j]) - __uint_as_float(c << 16);
            const float y1 = __uint_as_float(v[j + 1]) - __uint_as_float(c & 0xffff0000u);
            const float t0 = fold[q] + y0, t1 = fold[q + 1] + y1;
            comp2[q >> 1] = bf16x2_rn((t0 - fold[q]) - y0, (t1 - fold[q + 1]) - y1);
            fold[q] = t0;
            fold[q + 1] = t1;
        }
    }
}

// Output tile of a CTA: tile_m fastest over all tiles, or, for a symmetric
// product (A = B), the tiles on and above the diagonal only, column by column.
__device__ __forceinline__ void gram_tile(int idx, int tiles_m, bool sym, int& tm, int& tn) {
    if (!sym) {
        tm = idx % tiles_m;
        tn = idx / tiles_m;
        return;
    }
    tn = 0;
    while (idx > tn) {
        idx -= tn + 1;
        ++tn;
    }
    tm = idx;
}

template <bool ABS>
__global__ void __launch_bounds__(TW_THREADS, 1)
    tc_gram_ws_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, int M,
                      int N, size_t K, size_t kchunk, int tiles_m, bool sym, double* __restrict__ work,
                      int* __restrict__ err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint64_t full[TG2_STAGES], empty[TG2_STAGES], split_bar[2], mma_bar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int last_issued[TG2_STAGES];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* f32 = smem;
    unsigned char* bf = smem + TG2_STAGES * TG2_F32_STAGE;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tm, tn;
    gram_tile((int)blockIdx.x, tiles_m, sym, tm, tn);
    const int m0 = tm * TC_M, n0 = tn * TC_N;
    const size_t k_begin = (size_t)blockIdx.z * kchunk;
    const size_t k_end = min(K, k_begin + kchunk);
    const int nsteps = (int)((k_end - k_begin + TG2_BK - 1) / TG2_BK);
    const int nperiods = (nsteps + TG2_DRAIN - 1) / TG2_DRAIN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TG2_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TW_SPLIT_WARPS);
            last_issued[s] = -1;
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&split_bar[b], TW_SPLIT_WARPS);
            mbar_init(&mma_bar[b], 1);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        // two accumulators of 128 lanes x 128 FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    int committed = 0;  // MMA thread: steps committed

    if (warp == TW_SPLIT_WARPS) {
        // producer: step t into FP32 stage t % TG2_STAGES once its previous step was split
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
            for (int t = 0; t < nsteps; ++t) {
                const int s = t % TG2_STAGES;
                if (t >= TG2_STAGES &&
                    !mbar_wait_or_abort(&empty[s], (uint32_t)(t / TG2_STAGES - 1) & 1, &abort_sh))
                    break;
                const int x = (int)(k_begin + (size_t)t * TG2_BK);
                mbar_expect_tx(&full[s], TG2_F32_STAGE);
                tma_load_2d(f32 + s * TG2_F32_STAGE, &map_a, x, m0, &full[s]);
                tma_load_2d(f32 + s * TG2_F32_STAGE + TG2_F32_TILE, &map_b, x, n0, &full[s]);
                last_issued[s] = t;
            }
        }
    } else if (warp == TW_SPLIT_WARPS + 1) {
        // MMA issuer: step t accumulates into accumulator (t / TG2_DRAIN) mod 2,
        // starting it afresh at the first step of each period
        if (lane == 0) {
            for (int t = 0; t < nsteps; ++t) {
                const int b = t & 1;
                if (!mbar_wait_or_abort(&split_bar[b], (uint32_t)(t >> 1) & 1, &abort_sh)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a_hi = smem_u32(bf + b * TG2_BF_STAGE), a_lo = a_hi + TG2_BF_TILE;
                const uint32_t b_hi = a_hi + 2 * TG2_BF_TILE, b_lo = a_hi + 3 * TG2_BF_TILE;
                const uint32_t acc = tmem + (uint32_t)(((t / TG2_DRAIN) & 1) * TC_N);
#pragma unroll
                for (int kk = 0; kk < TG2_BK / 16; ++kk) {
                    const uint32_t ko = kk * 32;
                    const uint32_t first = (t % TG2_DRAIN == 0 && kk == 0) ? 0u : 1u;
                    mma_bf16(acc, sw64_desc(a_hi + ko), sw64_desc(b_hi + ko), first);
                    mma_bf16(acc, sw64_desc(a_hi + ko), sw64_desc(b_lo + ko), 1u);
                    mma_bf16(acc, sw64_desc(a_lo + ko), sw64_desc(b_hi + ko), 1u);
                    // |x| |x|: lo.lo >= 0 on the diagonal, so dropping it would bias it low
                    if (ABS) mma_bf16(acc, sw64_desc(a_lo + ko), sw64_desc(b_lo + ko), 1u);
                }
                mma_commit(&mma_bar[b]);
                committed = t + 1;
            }
        }
    } else {
        // splitters: 512 threads, TG2_VPT vectors per tile each; they also
        // drain period p once the MMAs of its last step, (p + 1) D - 1, are
        // done, i.e. at step t = (p + 1) D + 1 after the wait on mma[b] of
        // step t - 2, once step t is split.  The MMAs of period p + 2 (from
        // step (p + 2) D >= t + 1 for D >= 2) wait for the split[b] arrival
        // of that step, which follows the drain, so the accumulator is read
        // before they start it afresh.
        float fold[32];
        uint32_t comp2[16];
#pragma unroll
        for (int q = 0; q < 32; ++q) fold[q] = 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) comp2[q] = 0u;
        const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 32);
        int drained = 0;
        bool ok = true;
        for (int t = 0; t < nsteps; ++t) {
            const int s = t % TG2_STAGES, b = t & 1;
            if (!mbar_wait_or_abort(&full[s], (uint32_t)(t / TG2_STAGES) & 1, &abort_sh)) { ok = false; break; }
            // BF16 stage b: the MMAs of step t - 2 are done with it
            if (t >= 2 && !mbar_wait_or_abort(&mma_bar[b], (uint32_t)((t >> 1) - 1) & 1, &abort_sh)) {
                ok = false;
                break;
            }
            const unsigned char* fs = f32 + s * TG2_F32_STAGE;
            unsigned char* bs = bf + b * TG2_BF_STAGE;
            split_tile32<ABS>(fs, bs, bs + TG2_BF_TILE);
            split_tile32<ABS>(fs + TG2_F32_TILE, bs + 2 * TG2_BF_TILE, bs + 3 * TG2_BF_TILE);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[s]);
                mbar_arrive(&split_bar[b]);
            }
            // off the MMAs' path: the MMAs of step t (period p + 1) use the other accumulator
            if (t >= TG2_DRAIN + 1 && (t - 1) % TG2_DRAIN == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                drain_period(tlane + (uint32_t)((drained & 1) * TC_N), fold, comp2);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                ++drained;
            }
        }
        // the periods left: wait for the last step's commit (every MMA of this
        // CTA is then done; commits complete in issue order)
        if (ok && nsteps > 0 &&
            !mbar_wait_or_abort(&mma_bar[(nsteps - 1) & 1], (uint32_t)((nsteps - 1) >> 1) & 1, &abort_sh))
            ok = false;
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (; drained < nperiods; ++drained) drain_period(tlane + (uint32_t)((drained & 1) * TC_N), fold, comp2);
            const int row = m0 + (warp & 3) * 32 + lane;
            const int c0 = n0 + (warp >> 2) * 32;
            double* out = work + (size_t)blockIdx.z * M * N + (size_t)row * N;
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (c0 + q < N)
                        out[c0 + q] = (double)fold[q] -
                                      (double)__uint_as_float((q & 1) ? (comp2[q >> 1] & 0xffff0000u) : (comp2[q >> 1] << 16));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_sh) {
        // drain: copies still landing, MMAs still running (bounded waits)
        if (warp == TW_SPLIT_WARPS && lane == 0)
            for (int s = 0; s < TG2_STAGES; ++s)
                if (last_issued[s] >= 0) mbar_wait(&full[s], (uint32_t)(last_issued[s] / TG2_STAGES) & 1);
        if (warp == TW_SPLIT_WARPS + 1 && lane == 0 && committed > 0)
            mbar_wait(&mma_bar[(committed - 1) & 1], (uint32_t)((committed - 1) >> 1) & 1);
        if (threadIdx.x == 0) atomicExch(err, 1);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

// Sum of the chunks in FP64 in a fixed order; for a symmetric product the
// tiles below the diagonal were not computed and are read mirrored.
__global__ void tc_reduce_kernel(int M, int N, int nchunk, const double* __restrict__ work, double alpha, bool sym,
                                 double* __restrict__ C, int ldc) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)M * N) return;
    const int m = (int)(idx / N), n = (int)(idx % N);
    const size_t src = (sym && n / TC_N < m / TC_M) ? (size_t)n * N + m : idx;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += work[(size_t)c * M * N + src];
    C[(size_t)m * ldc + n] = alpha * s;
}

// ---------------------------------------------------------------------------
// Combination over orbitals: Out[n][r] = beta Out[n][r] + sum_k Coef[k][n] A[k][r]
// (xi = W L^{-T}; K_ACE psi = -xi X).  As an MMA: D[r][n] = sum_k A^T[r][k]
// Coef[k][n], M = 128 grid points per CTA, N = 256 target orbitals, K = the
// orbitals being combined (64 per step).  The A tile is transposed while it is
// staged (each thread loads 4 consecutive k of one r and stores one 8-byte
// chunk of the K-major row r); Coef is pre-split into BF16 hi/lo rows
// CoefT[n][k] once per call.
constexpr int CB_N = 256;
constexpr int CB_A_BYTES = TC_M * TC_BK * 2;   // 16 KB
constexpr int CB_B_BYTES = CB_N * TC_BK * 2;   // 32 KB
constexpr int CB_STAGE_BYTES = 2 * CB_A_BYTES + 2 * CB_B_BYTES;
constexpr int CB_SMEM_BYTES = 2 * CB_STAGE_BYTES + 1024;
constexpr uint32_t kIdescN256 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CB_N >> 3) << 17) |
                                ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ void mma_bf16_n256(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescN256), "r"(accumulate));
}

// hiT[n][k], loT[n][k] (BF16, rows of kpad, zero padded) from Coef[k][n] (FP64)
__global__ void coef_split_kernel(int Kc, int N, const double* __restrict__ coef, int ldcoef, int kpad, int npad,
                                  __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= npad * kpad) return;
    const int n = idx / kpad, k = idx % kpad;
    const float x = (n < N && k < Kc) ? (float)coef[(size_t)k * ldcoef + n] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hiT[idx] = h;
    loT[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}

template <typename TO>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_combine_kernel(int N, size_t K, int Kc, int kpad, const float* __restrict__ A, size_t lda,
                      const __nv_bfloat16* __restrict__ hiT, const __nv_bfloat16* __restrict__ loT, float beta,
                      TO* __restrict__ Out, size_t ldo, int* __restrict__ err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5;
    const size_t r0 = (size_t)blockIdx.x * TC_M;
    const int n0 = blockIdx.y * CB_N;
    const int nsteps = kpad / TC_BK;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(CB_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    // this thread stages grid point r = tid % 128 and k-quads q = tid / 128 + 4j
    const int ar = threadIdx.x & (TC_M - 1), aq = threadIdx.x >> 7;
    const bool rvalid = r0 + ar < K;
    uint32_t uses[2] = {0u, 0u};
    for (int step = 0; step < nsteps; ++step) {
        const int s = step & 1;
        unsigned char* st = smem + s * CB_STAGE_BYTES;
        if (uses[s] > 0) {
            if (threadIdx.x == 0 && !mbar_wait(&bars[s], (uses[s] - 1) & 1)) abort_sh = 1;
            __syncthreads();
            if (abort_sh) break;
        }
        const int k0 = step * TC_BK;
        // A^T tile: 128 r x 64 k, 16 quads of 4 k per row, 4 per thread
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kq = (aq + 4 * j) * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (rvalid) {
                const int k = k0 + kq;
                const float* p = A + (size_t)k * lda + r0 + ar;
                if (k + 0 < Kc) v.x = __ldg(p);
                if (k + 1 < Kc) v.y = __ldg(p + lda);
                if (k + 2 < Kc) v.z = __ldg(p + 2 * lda);
                if (k + 3 < Kc) v.w = __ldg(p + 3 * lda);
            }
            uint2 h, l;
            split4(v, h, l);
            const uint32_t off = sw128_off(ar, kq);
            *reinterpret_cast<uint2*>(st + off) = h;
            *reinterpret_cast<uint2*>(st + CB_A_BYTES + off) = l;
        }
        // B tiles: rows n0.., 64 k of the pre-split CoefT (16-byte chunks)
        {
            unsigned char* bh = st + 2 * CB_A_BYTES;
            unsigned char* bl = bh + CB_B_BYTES;
#pragma unroll
            for (int j = 0; j < (CB_N * 8) / TC_THREADS; ++j) {
                const int e = threadIdx.x + j * TC_THREADS;
                const int n = e >> 3, c = e & 7;
                const size_t g = (size_t)(n0 + n) * kpad + k0 + c * 8;
                const uint4 hv = *reinterpret_cast<const uint4*>(hiT + g);
                const uint4 lv = *reinterpret_cast<const uint4*>(loT + g);
                const uint32_t off = (uint32_t)(n * 128 + (((c ^ (n & 7)) & 7) << 4));
                *reinterpret_cast<uint4*>(bh + off) = hv;
                *reinterpret_cast<uint4*>(bl + off) = lv;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(st), a_lo = a_hi + CB_A_BYTES;
            const uint32_t b_hi = a_hi + 2 * CB_A_BYTES, b_lo = b_hi + CB_B_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint32_t ko = kk * 32;
                const uint32_t first = (step == 0 && kk == 0) ? 0u : 1u;
                mma_bf16_n256(tmem, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), first);
                mma_bf16_n256(tmem, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), 1u);
                mma_bf16_n256(tmem, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), 1u);
            }
            mma_commit(&bars[s]);
        }
        uses[s] += 1;
    }
    if (nsteps > 0 && !abort_sh) {
        const int s = (nsteps - 1) & 1;
        if (threadIdx.x == 0 && !mbar_wait(&bars[s], (uses[s] - 1) & 1)) abort_sh = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_sh) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else if (warp < 4) {
        const size_t r = r0 + warp * 32 + (threadIdx.x & 31);
#pragma unroll 1
        for (int c0 = 0; c0 < CB_N; c0 += 16) {
            if (n0 + c0 >= N) break;
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < K) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) {
                        TO* o = Out + (size_t)n * ldo + r;
                        *o = beta == 0.f ? (TO)__uint_as_float(v[j]) : (TO)(beta * (float)*o + __uint_as_float(v[j]));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB_N) : "memory");
    }
}

// The combination with its operands brought in by the Tensor Memory
// Accelerator, persistent over output tiles: each CTA takes tiles (128 grid
// points x 256 targets) round-robin and runs their 64-orbital steps as one
// pipeline of TC_STAGES-deep copies: per step, the FP32 A tile [64 k][128 r]
// (row-major, rows past Kc and columns past K arrive as zeros) and the
// pre-split Coef^T hi/lo tiles [256 n][64 k], which TMA writes directly in
// the 128-byte swizzled K-major layout the MMA reads.  All 512 threads
// transpose-split A into the BF16 hi/lo tiles (one BF16 stage: the split of a
// step waits for the MMAs of the step before, and a stage's copies are
// replaced only after its MMAs are done); after a tile's last MMA all 16
// warps read the accumulators (warp w: lanes 32 (w % 4).., columns 64 (w / 4)..)
// and write Out.  Bounded waits throughout; on a timeout the CTA records an
// error, waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and returns.
constexpr int CT_STAGES = 2;
constexpr int CT_A32_BYTES = TC_BK * TC_M * 4;                 // 32 KB: 64 k x 128 r FP32
constexpr int CT_STAGE_BYTES = CT_A32_BYTES + 2 * CB_B_BYTES;  // + Coef^T hi, lo (32 KB each)
constexpr int CT_SMEM_BYTES = CT_STAGES * CT_STAGE_BYTES + 2 * CB_A_BYTES + 1024;

template <typename TO>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_combine_tma_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_hi,
                          const __grid_constant__ CUtensorMap map_lo, int N, size_t K, int kpad, float beta,
                          TO* __restrict__ Out, size_t ldo, int* __restrict__ err) {
    extern __shared__ unsigned char tc_smem_raw[];
    __shared__ uint64_t full[CT_STAGES];
    __shared__ uint64_t mma_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* abf = smem + CT_STAGES * CT_STAGE_BYTES;  // A^T hi, lo (swizzled K-major, 128 rows r)
    const int warp = threadIdx.x >> 5;
    const int nsteps = kpad / TC_BK;
    const int rtiles = (int)((K + TC_M - 1) / TC_M), ntiles = (N + CB_N - 1) / CB_N;
    const int tiles = rtiles * ntiles;
    const int my_tiles = blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * nsteps;  // this CTA's steps over all its tiles
    if (threadIdx.x == 0) {
        for (int s = 0; s < CT_STAGES; ++s) mbar_init(&full[s], 1);
        mbar_init(&mma_bar, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_hi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_lo)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(CB_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    // thread 0: global step g (tile g / nsteps of this CTA, orbital step g % nsteps) into stage g % CT_STAGES
    int issued = 0;
    auto issue = [&](int g) {
        const int s = g % CT_STAGES;
        const int tile = (int)blockIdx.x + (g / nsteps) * (int)gridDim.x;
        const int rt = tile % rtiles, nt = tile / rtiles;
        const int k0 = (g % nsteps) * TC_BK;
        unsigned char* st = smem + s * CT_STAGE_BYTES;
        mbar_expect_tx(&full[s], CT_STAGE_BYTES);
        tma_load_2d(st, &map_a, rt * TC_M, k0, &full[s]);
        tma_load_2d(st + CT_A32_BYTES, &map_hi, k0, nt * CB_N, &full[s]);
        tma_load_2d(st + CT_A32_BYTES + CB_B_BYTES, &map_lo, k0, nt * CB_N, &full[s]);
    };
    if (threadIdx.x == 0)
        for (; issued < CT_STAGES && issued < total; ++issued) issue(issued);
    // this thread's transpose-split share: grid point ar, k quads aq + 4j
    const int ar = threadIdx.x & (TC_M - 1), aq = threadIdx.x >> 7;
    int g = 0, committed = 0;
    for (; g < total; ++g) {
        const int s = g % CT_STAGES, step = g % nsteps;
        bool ok = mbar_wait(&full[s], (uint32_t)(g / CT_STAGES) & 1);
        if (g > 0) ok = ok && mbar_wait(&mma_bar, (uint32_t)(g - 1) & 1);
        if (!ok) abort_sh = 1;
        __syncthreads();
        if (abort_sh) break;
        // the MMAs of step g - 1 are done: its stage may be refilled
        if (threadIdx.x == 0 && g > 0 && issued < total) issue(issued++);
        if (g > 0 && step == 0) {
            // the previous tile is complete: accumulators -> Out
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int tile = (int)blockIdx.x + ((g - 1) / nsteps) * (int)gridDim.x;
            const int rt = tile % rtiles, nt = tile / rtiles;
            const size_t r = (size_t)rt * TC_M + (warp & 3) * 32 + (threadIdx.x & 31);
            const int cb = (warp >> 2) * 64;
#pragma unroll 1
            for (int c0 = cb; c0 < cb + 64; c0 += 16) {
                if (nt * CB_N + c0 >= N) break;
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (r < K) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = nt * CB_N + c0 + j;
                        if (n < N) {
                            TO* o = Out + (size_t)n * ldo + r;
                            *o = beta == 0.f ? (TO)__uint_as_float(v[j]) : (TO)(beta * (float)*o + __uint_as_float(v[j]));
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        // A^T: FP32 [64 k][128 r] -> BF16 hi/lo, K-major rows r
        const float* a32 = reinterpret_cast<const float*>(smem + s * CT_STAGE_BYTES);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int kq = (aq + 4 * j) * 4;
            const float4 v = make_float4(a32[(kq + 0) * TC_M + ar], a32[(kq + 1) * TC_M + ar],
                                         a32[(kq + 2) * TC_M + ar], a32[(kq + 3) * TC_M + ar]);
            uint2 h, l;
            split4(v, h, l);
            const uint32_t off = sw128_off(ar, kq);
            *reinterpret_cast<uint2*>(abf + off) = h;
            *reinterpret_cast<uint2*>(abf + CB_A_BYTES + off) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(abf), a_lo = a_hi + CB_A_BYTES;
            const uint32_t b_hi = smem_u32(smem + s * CT_STAGE_BYTES + CT_A32_BYTES), b_lo = b_hi + CB_B_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint32_t ko = kk * 32;
                const uint32_t first = (step == 0 && kk == 0) ? 0u : 1u;
                mma_bf16_n256(tmem, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), first);
                mma_bf16_n256(tmem, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), 1u);
                mma_bf16_n256(tmem, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), 1u);
            }
            mma_commit(&mma_bar);
        }
        committed = g + 1;
    }
    if (threadIdx.x == 0) {
        if (abort_sh) {
            for (int t = g; t < issued; ++t) mbar_wait(&full[t % CT_STAGES], (uint32_t)(t / CT_STAGES) & 1);
            if (committed > 0) mbar_wait(&mma_bar, (uint32_t)(committed - 1) & 1);
        } else if (total > 0 && !mbar_wait(&mma_bar, (uint32_t)(total - 1) & 1)) {
            abort_sh = 1;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_sh) {
        if (threadIdx.x == 0) atomicExch(err, 1);
    } else if (total > 0) {
        // the last tile
        const int tile = (int)blockIdx.x + ((total - 1) / nsteps) * (int)gridDim.x;
        const int rt = tile % rtiles, nt = tile / rtiles;
        const size_t r = (size_t)rt * TC_M + (warp & 3) * 32 + (threadIdx.x & 31);
        const int cb = (warp >> 2) * 64;
#pragma unroll 1
        for (int c0 = cb; c0 < cb + 64; c0 += 16) {
            if (nt * CB_N + c0 >= N) break;
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < K) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = nt * CB_N + c0 + j;
                    if (n < N) {
                        TO* o = Out + (size_t)n * ldo + r;
                        *o = beta == 0.f ? (TO)__uint_as_float(v[j]) : (TO)(beta * (float)*o + __uint_as_float(v[j]));
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CB_N) : "memory");
    }
}

}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder (through the runtime's entry-point query,
// so no link against the driver library), or null.  LACE_TC_TMA=0 turns the
// TMA-fed Gram kernel off (tuning: the register-staged kernel then runs).
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        const char* e = getenv("LACE_TC_TMA");
        if (e && e[0] == '0') return nullptr;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor map of a row-major matrix [rows][cols] (row pitch ld elements of
// esize bytes; 16-byte aligned base and pitch) in boxes of box_rows x
// box_cols; reads outside the matrix return zeros.
bool make_map(CUtensorMap* m, CUtensorMapDataType type, size_t esize, const void* base, size_t rows, size_t cols,
              size_t ld, int box_cols, int box_rows, CUtensorMapSwizzle swz) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || rows == 0 || cols == 0 || rows > 0xffffffffull || cols > 0xffffffffull) return false;
    if (((uintptr_t)base % 16) || ((ld * esize) % 16)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * esize)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// FP32 [rows][cols] in boxes of 128 rows x bk columns (the Gram's A and B tiles).
bool make_tile_map(CUtensorMap* m, const float* base, size_t rows, size_t cols, size_t ld, int bk) {
    return make_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), base, rows, cols, ld, bk, TC_M,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
}


}  // namespace

size_t tc_combine_scratch_bytes(int N, int Kc) {
    const size_t kpad = ((size_t)Kc + TC_BK - 1) / TC_BK * TC_BK;
    const size_t npad = ((size_t)N + CB_N - 1) / CB_N * CB_N;
    return 2 * kpad * npad * sizeof(__nv_bfloat16);
}

template <typename TO>
cudaError_t tc_combine(int N, size_t K, int Kc, const float* A, size_t lda, const double* Coef, int ldcoef,
                       double beta, TO* Out, size_t ldo, void* scratch, int* d_err, int* h_err, cudaStream_t s,
                       int* launches) {
    if (N <= 0 || K == 0) return cudaSuccess;
    const int kpad = (Kc + TC_BK - 1) / TC_BK * TC_BK;
    const int npad = (N + CB_N - 1) / CB_N * CB_N;
    __nv_bfloat16* hiT = static_cast<__nv_bfloat16*>(scratch);
    __nv_bfloat16* loT = hiT + (size_t)kpad * npad;
    static std::atomic<unsigned long long> attr_done{0};  // one per output type
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !(attr_done.load() & (1ull << dev))) {
        cudaError_t e =
            cudaFuncSetAttribute(tc_combine_kernel<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, CB_SMEM_BYTES);
        if (!e)
            e = cudaFuncSetAttribute(tc_combine_tma_kernel<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     CT_SMEM_BYTES);
        if (e) return e;
        attr_done.fetch_or(1ull << dev);
    }
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    const int tot = kpad * npad;
    coef_split_kernel<<<(tot + 255) / 256, 256, 0, s>>>(Kc, N, Coef, ldcoef, kpad, npad, hiT, loT);
    // TMA-fed persistent kernel: A as [Kc][K] FP32 in boxes of 64 k x 128 r;
    // Coef^T hi/lo as [npad][kpad] BF16 in boxes of 256 n x 64 k, written by
    // the copy in the 128-byte swizzled layout
    CUtensorMap map_a, map_hi, map_lo;
    const bool tma = K <= 0x7fffffffull &&
                     make_map(&map_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), A, (size_t)Kc, K, lda, TC_M,
                              TC_BK, CU_TENSOR_MAP_SWIZZLE_NONE) &&
                     make_map(&map_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, hiT, (size_t)npad, (size_t)kpad,
                              (size_t)kpad, TC_BK, CB_N, CU_TENSOR_MAP_SWIZZLE_128B) &&
                     make_map(&map_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, loT, (size_t)npad, (size_t)kpad,
                              (size_t)kpad, TC_BK, CB_N, CU_TENSOR_MAP_SWIZZLE_128B);
    if (tma) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long tiles = (long long)((K + TC_M - 1) / TC_M) * (npad / CB_N);
        const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(tiles, sms));
        tc_combine_tma_kernel<TO><<<grid, TC_THREADS, CT_SMEM_BYTES, s>>>(map_a, map_hi, map_lo, N, K, kpad,
                                                                          (float)beta, Out, ldo, d_err);
    } else {
        dim3 grid((unsigned)((K + TC_M - 1) / TC_M), npad / CB_N);
        tc_combine_kernel<TO><<<grid, TC_THREADS, CB_SMEM_BYTES, s>>>(N, K, Kc, kpad, A, lda, hiT, loT,
                                                                      (float)beta, Out, ldo, d_err);
    }
    *launches += 2;
    if (h_err) {
        cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return e;
    }
    return cudaGetLastError();
}


namespace {
// Output tiles of the Gram (only those on and above the diagonal when symmetric).
size_t gram_tiles(int M, int N, bool sym) {
    const size_t tm = (M + TC_M - 1) / TC_M, tn = (N + TC_N - 1) / TC_N;
    return sym ? tm * (tm + 1) / 2 : tm * tn;
}
// K chunks: as many CTAs as fit one wave of 152 SMs (one CTA per SM), a
// chunk at least 4096 points long.
size_t gram_chunks(int M, int N, size_t K, bool sym) {
    const size_t tiles = gram_tiles(M, N, sym);
    const size_t want = std::max<size_t>(1, 152 / tiles);
    const size_t maxc = (K + 4095) / 4096;
    return std::max<size_t>(1, std::min(want, maxc));
}
}  // namespace

size_t tc_gram_work_elems(int M, int N, size_t K, bool sym) { return gram_chunks(M, N, K, sym) * (size_t)M * N; }

cudaError_t tc_gram(int M, int N, size_t K, const float* A, size_t lda, const float* B, size_t ldb, double alpha,
                    double* C, int ldc, double* work, size_t work_elems, int* d_err, int* h_err, cudaStream_t s,
                    int* launches, bool absval, bool sym) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // 16-byte row alignment for the vector loads
    if ((lda % 4) || (ldb % 4) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16)) return cudaErrorInvalidValue;
    if (sym && (A != B || M != N || lda != ldb)) return cudaErrorInvalidValue;
    const size_t nch = gram_chunks(M, N, K, sym);
    if (nch * (size_t)M * N > work_elems) return cudaErrorInvalidValue;
    size_t kchunk = (K + nch - 1) / nch;
    kchunk = (kchunk + TC_BK - 1) / TC_BK * TC_BK;
    const size_t nch_eff = (K + kchunk - 1) / kchunk;
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !(attr_done.load() & (1ull << dev))) {
        cudaError_t e = cudaSuccess;
        for (auto f : {tc_gram_kernel<false>, tc_gram_kernel<true>})
            if (!e) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
        for (auto f : {tc_gram_ws_kernel<false>, tc_gram_ws_kernel<true>})
            if (!e) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, TG2_SMEM_BYTES);
        if (e) return e;
        attr_done.fetch_or(1ull << dev);
    }
    cudaMemsetAsync(d_err, 0, sizeof(int), s);
    const int tiles_m = (M + TC_M - 1) / TC_M;
    CUtensorMap map_a, map_b;
    bool mirrored = false;
    if (K <= 0x7fffffffull && make_tile_map(&map_a, A, (size_t)M, K, lda, TG2_BK) &&
        make_tile_map(&map_b, B, (size_t)N, K, ldb, TG2_BK)) {
        dim3 grid((unsigned)gram_tiles(M, N, sym), 1, (unsigned)nch_eff);
        auto kern = absval ? tc_gram_ws_kernel<true> : tc_gram_ws_kernel<false>;
        kern<<<grid, TW_THREADS, TG2_SMEM_BYTES, s>>>(map_a, map_b, M, N, K, kchunk, tiles_m, sym, work, d_err);
        mirrored = sym;
    } else {
        dim3 grid(tiles_m, (N + TC_N - 1) / TC_N, (unsigned)nch_eff);
        auto kern = absval ? tc_gram_kernel<true> : tc_gram_kernel<false>;
        kern<<<grid, TC_THREADS, TC_SMEM_BYTES, s>>>(M, N, K, A, lda, B, ldb, kchunk, work, d_err);
    }
    const size_t tot = (size_t)M * N;
    tc_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, N, (int)nch_eff, work, alpha, mirrored, C, ldc);
    *launches += 2;
    if (h_err) {
        cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) return e;
    }
    return cudaGetLastError();
}

template cudaError_t tc_combine<float>(int, size_t, int, const float*, size_t, const double*, int, double, float*,
                                       size_t, void*, int*, int*, cudaStream_t, int*);
template cudaError_t tc_combine<double>(int, size_t, int, const float*, size_t, const double*, int, double, double*,
                                        size_t, void*, int*, int*, cudaStream_t, int*);

}  // namespace lace
