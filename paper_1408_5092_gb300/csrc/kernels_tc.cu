// Split-bfloat16 (or split-float16) grouped block GEMM on the 5th-generation
// tensor cores (tcgen05, sm_103a).  Same task lists as the float64 kernel:
// each CTA owns one 128 x 64 output tile and walks its K-list; every float64
// operand value v is split into hi = bf16(v), lo = bf16(v - hi) (f16 in the
// float16 variant) while it is staged into shared memory, and the tile
// accumulates Ahi*Bhi + Ahi*Blo + Alo*Bhi in float32 in tensor memory (TMEM).  One elected thread issues the MMAs and
// commits them to an mbarrier per shared-memory stage (double buffered).
// The eight warps stage the operands with 16 independent loads in flight
// per thread, and read the accumulator back with tcgen05.ld (warp w: TMEM
// lanes 32 (w mod 4) .. +31, columns 32 (w / 4) .. +31).
//
// Shared-memory operand layout: K-major, no swizzle, 8x8 core matrices
// (8 rows x 16 bytes); byte offset of (row r, k) inside a 64-wide K stage:
//   (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// so the leading-dimension (K) core-matrix stride is 128 B and the
// stride-dimension (8-row group) stride is 1024 B.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.h"

namespace mpspt {
namespace {

constexpr int BM = 128;     // tcgen05 M (cta_group::1)
constexpr int BN = 64;      // tcgen05 N
constexpr int BK = 64;      // K per shared-memory stage
constexpr int NTH = 256;    // 8 warps
constexpr int LCH = 16;     // operand loads in flight per thread
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // hi + lo of A and B
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 64;
constexpr long long WAIT_LIMIT = 1LL << 26;              // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// tcgen05 shared-memory matrix descriptor (K-major, SWIZZLE_NONE).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;    // leading dimension (K) byte offset
    d |= (uint64_t)(1024 >> 4) << 32;   // stride dimension (8-row group) byte offset
    d |= (uint64_t)1 << 46;             // descriptor version (tcgen05)
    return d;                            // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B of the
// same 16-bit type (bits 7-9 and 10-12: 1 = bf16, 0 = f16), both K-major.
template <bool F16>
__host__ __device__ constexpr uint32_t make_idesc() {
    return (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(bar)));
}

// float64 -> float32, round to nearest even, with integer operations only
// (the float64 pipe of this GPU is narrow: the conversion instruction would
// bound the operand staging).  Magnitudes below the float32 normal range
// (2^-126) become signed zero, above it infinity; NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
    const int fe = e - 1023 + 127;
    if (fe <= 0) return __uint_as_float(sign);
    if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    const unsigned mant = (unsigned)(m >> 29);
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFULL);
    unsigned f = sign | ((unsigned)fe << 23) | mant;
    if (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) f += 1u;   // carry may reach the exponent
    return __uint_as_float(f);
}

// hi = round(f), lo = round(f - hi) in the 16-bit type (bf16 or f16)
template <bool F16>
__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, uint32_t off, float f) {
    if constexpr (F16) {
        const __half h = __float2half_rn(f);
        const __half l = __float2half_rn(f - __half2float(h));
        *reinterpret_cast<__half*>(hi + off) = h;
        *reinterpret_cast<__half*>(lo + off) = l;
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(f);
        const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
    }
}

// Persistent: at most the resident CTAs are launched; CTA b takes tasks b,
// b + gridDim.x, ... with one TMEM allocation and one barrier pair for all of
// them (the stage counter, and with it the mbarrier phases, runs on across
// tasks).
template <bool F16>
__global__ void __launch_bounds__(NTH, 1) k_gemm_tc(const GemmTask* __restrict__ tasks, int ntask,
                                                    const GemmOp* __restrict__ ops, int* err,
                                                    const int* __restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int wait_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base_sh;
    constexpr uint32_t idesc = make_idesc<F16>();

    int stage = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntask && ok; ti += gridDim.x) {
        const GemmTask t = tasks[ti];
        const int mrem = min(BM, t.m - t.r0);
        const int nrem = min(BN, t.n - t.c0);
        const int stage0 = stage;
        int kbase = 0;   // position of op o's first K index in the task's concatenated K-list
        for (int o = t.op0; o < t.op1 && ok; ++o) {
            const GemmOp op = ops[o];
            const int kb = max(0, t.kb - kbase), ke = min(op.k, t.ke - kbase);
            kbase += op.k;
            if (kb >= ke) continue;
            const bool ta = op.trans & 1, tb = op.trans & 2;
            const float alpha = d2f_rn(op.alpha);
            for (int k0 = kb; k0 < ke; k0 += BK) {
                const int buf = stage & 1;
                if (stage >= 2) {   // stage buffer free once the MMAs of stage-2 completed
                    if (tid == 0) wait_ok = mbar_wait(&bars[buf], ((stage - 2) >> 1) & 1) ? 1 : 0;
                    __syncthreads();
                    if (!wait_ok) { ok = false; break; }
                }
                unsigned char* Ahi = smem + buf * STAGE_BYTES;
                unsigned char* Alo = Ahi + A_BYTES;
                unsigned char* Bhi = Alo + A_BYTES;
                unsigned char* Blo = Bhi + B_BYTES;
                const int krem = min(BK, ke - k0);
                // A: BM x BK values, B: BN x BK values; LCH loads per thread are
                // issued before any of them is split and stored
                for (int e0 = 0; e0 < BM * BK; e0 += NTH * LCH) {
                    double v[LCH];
                    int off[LCH];
#pragma unroll
                    for (int q = 0; q < LCH; ++q) {
                        const int e = e0 + q * NTH + tid;
                        int r, kk;
                        if (ta) { r = e % BM; kk = e / BM; } else { kk = e % BK; r = e / BK; }
                        off[q] = (int)tile_off(r, kk);
                        v[q] = 0.0;
                        if (r < mrem && kk < krem) {
                            const int row = t.r0 + r, kg = k0 + kk;
                            v[q] = ta ? op.A[(size_t)kg * op.lda + row] : op.A[(size_t)row * op.lda + kg];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < LCH; ++q)
                        split_store<F16>(Ahi, Alo, (uint32_t)off[q], alpha * d2f_rn(v[q]));
                }
                for (int e0 = 0; e0 < BN * BK; e0 += NTH * LCH) {
                    double v[LCH];
                    int off[LCH];
#pragma unroll
                    for (int q = 0; q < LCH; ++q) {
                        const int e = e0 + q * NTH + tid;
                        int j, kk;
                        if (tb) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
                        off[q] = (int)tile_off(j, kk);
                        v[q] = 0.0;
                        if (j < nrem && kk < krem) {
                            const int col = t.c0 + j, kg = k0 + kk;
                            v[q] = tb ? op.B[(size_t)col * op.ldb + kg] : op.B[(size_t)kg * op.ldb + col];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < LCH; ++q) split_store<F16>(Bhi, Blo, (uint32_t)off[q], d2f_rn(v[q]));
                }
                asm volatile("fence.proxy.async.shared::cta;");
                __syncthreads();
                if (tid == 0) {
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
                    const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
                    for (int j = 0; j < BK / 16; ++j) {
                        const uint32_t kofs = j * 256;   // two 128-byte core matrices per 16 K
                        mma_bf16(tmem, make_desc(ahi + kofs), make_desc(bhi + kofs), idesc,
                                 (stage > stage0 || j > 0) ? 1u : 0u);
                        mma_bf16(tmem, make_desc(ahi + kofs), make_desc(blo + kofs), idesc, 1u);
                        mma_bf16(tmem, make_desc(alo + kofs), make_desc(bhi + kofs), idesc, 1u);
                    }
                    mma_commit(&bars[buf]);
                }
                ++stage;
            }
        }
        const bool any = stage > stage0;
        if (any && ok) {
            if (tid == 0) wait_ok = mbar_wait(&bars[(stage - 1) & 1], ((stage - 1) >> 1) & 1) ? 1 : 0;
            __syncthreads();
            ok = wait_ok != 0;
        }
        if (!ok) {
            if (tid == 0) {
                atomicExch(err, 1);
                // give in-flight MMAs a bounded chance to drain before releasing TMEM
                if (stage > 0) mbar_wait(&bars[(stage - 1) & 1], ((stage - 1) >> 1) & 1);
            }
            __syncthreads();
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (accumulator
        // rows), columns 32 (w / 4) .. +31
        const int row = (warp & 3) * 32 + lane;
#pragma unroll 1
        for (int c0 = (warp >> 2) * 32; c0 < (warp >> 2) * 32 + 32; c0 += 16) {
            uint32_t v[16];
            if (any && ok) {
                const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0u;
            }
            if (row < mrem && ok) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = c0 + q;
                    if (col < nrem && t.part) {   // split-K partial tile (BM x BN, row-major)
                        t.part[row * BN + col] = (double)__uint_as_float(v[q]);
                    } else if (col < nrem) {
                        const int gr = t.r0 + row, gc = t.c0 + col;
                        double* dst;
                        if (t.cmap == nullptr) dst = t.C + (size_t)gr * t.ldc + gc;
                        else if (t.cmap_rows) dst = t.C + t.cmap[2 * gr] + (size_t)gc * t.cmap[2 * gr + 1];
                        else dst = t.C + t.cmap[2 * gc] + (size_t)gr * t.cmap[2 * gc + 1];
                        const double val = (double)__uint_as_float(v[q]);
                        *dst = t.accumulate ? *dst + val : val;
                    }
                }
            }
        }
        // the next task's first MMA overwrites the accumulator: every warp's
        // tcgen05.ld above completes before it (wait::ld, then this barrier)
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

// Resident CTAs of the kernel on the current device, per (kernel, device).
int tc_resident_ctas(const void* f) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    thread_local std::map<std::pair<const void*, int>, int> mine;   // lock-free fast path per thread
    int dev = 0;
    cudaGetDevice(&dev);
    auto g = mine.find({f, dev});
    if (g != mine.end()) return g->second;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find({f, dev});
    if (it != cache.end()) return mine[{f, dev}] = it->second;
    int nb = 1, sms = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, NTH, SMEM_BYTES) != cudaSuccess || nb < 1) nb = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    cudaGetLastError();
    return mine[{f, dev}] = cache[{f, dev}] = nb * sms;
}

int tc_tile_m() { return BM; }
int tc_tile_n() { return BN; }

void launch_gemm_tc(const GemmTask* tasks, int ntask, const GemmOp* ops, int* err, cudaStream_t st,
                    const int* skip, bool f16) {
    if (ntask <= 0) return;
    count_launch();
    const void* f = f16 ? reinterpret_cast<const void*>(k_gemm_tc<true>) : reinterpret_cast<const void*>(k_gemm_tc<false>);
    ensure_smem_attr(f, SMEM_BYTES);
    const int grid = std::min(ntask, tc_resident_ctas(f));
    if (f16) k_gemm_tc<true><<<grid, NTH, SMEM_BYTES, st>>>(tasks, ntask, ops, err, skip);
    else k_gemm_tc<false><<<grid, NTH, SMEM_BYTES, st>>>(tasks, ntask, ops, err, skip);
}

}  // namespace mpspt
