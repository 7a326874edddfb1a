// BF16 GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] (fp32) =
// op(A) op(B), op(A)(m,k) = ta ? A[k*lda+m] : A[m*lda+k],
// op(B)(k,n) = tb ? B[n*ldb+k] : B[k*ldb+n] (bf16, row-major).
//
// One CTA of 128 threads per 128 x 128 tile of C; K in steps of 64. The
// threads stage both operand tiles into shared memory in the canonical
// K-major, non-swizzled layout of the tensor-core descriptors (8 x 8 core
// matrices of 16-byte rows, 128 bytes each; core matrices adjacent in K are
// 128 bytes apart, those adjacent in M/N 1024 bytes apart), zero-filling past
// the edges, so any transposition and any M, N, K are handled in the copy.
// One elected thread issues four tcgen05.mma (M = 128, N = 128, K = 16 each)
// per K step into an FP32 accumulator in tensor memory and commits them to an
// mbarrier that every thread waits on (bounded) before the tiles are
// overwritten. The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes 32w..32w+31 = rows of the tile) and stores the valid part of C.
// A wait that runs out of iterations sets *err, waits once more (bounded) for
// the MMAs in flight, frees the tensor memory and returns.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace pimd {

constexpr int UMMA_M = 128, UMMA_N = 128, UMMA_K = 64;
constexpr uint32_t UMMA_TMEM_COLS = 128;
constexpr long long UMMA_WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t umma_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, the fixed 0b001 field at bits 46-48, base offset 0,
// no swizzling
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool umma_wait(uint32_t bar, uint32_t phase)
{
    for (long long it = 0; it < UMMA_WAIT_LIMIT; it++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// offset (in elements) of tile element (row, k) in the core-matrix layout
__device__ __forceinline__ int umma_tile_off(int row, int k)
{
    return (((row >> 3) * (UMMA_K / 8) + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

__global__ void __launch_bounds__(128) bf16_gemm_tc_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                           int lda, int ta, const __nv_bfloat16* __restrict__ B,
                                                           int ldb, int tb, float* __restrict__ C, int ldc, int* err)
{
    __shared__ __align__(1024) __nv_bfloat16 sA[UMMA_M * UMMA_K];
    __shared__ __align__(1024) __nv_bfloat16 sB[UMMA_N * UMMA_K];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int m0 = blockIdx.y * UMMA_M, n0 = blockIdx.x * UMMA_N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t bar_a = umma_smem_addr(&bar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         umma_smem_addr(&tmem_slot)),
                     "r"(UMMA_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = umma_idesc_bf16(UMMA_M, UMMA_N);
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    uint32_t phase = 0;
    bool ok = true;
    const int nk = (K + UMMA_K - 1) / UMMA_K;
    for (int kt = 0; kt < nk && ok; kt++) {
        const int k0 = kt * UMMA_K;
        // 128 rows x 64 k per tile: thread t copies rows t (A) and t (B)
        {
            const int r = threadIdx.x;
            const int m = m0 + r, n = n0 + r;
#pragma unroll 4
            for (int kk = 0; kk < UMMA_K; kk++) {
                const int k = k0 + kk;
                const bool kin = k < K;
                sA[umma_tile_off(r, kk)] =
                    (kin && m < M) ? (ta ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : z;
                sB[umma_tile_off(r, kk)] =
                    (kin && n < N) ? (tb ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]) : z;
            }
        }
        // generic-proxy writes of the tiles -> visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < UMMA_K / 16; kk++) {
                const uint64_t ad = umma_smem_desc(umma_smem_addr(sA) + kk * 256, 128, (UMMA_K / 8) * 128);
                const uint64_t bd = umma_smem_desc(umma_smem_addr(sB) + kk * 256, 128, (UMMA_K / 8) * 128);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                         : "memory");
        }
        ok = umma_wait(bar_a, phase);
        phase ^= 1u;
        // every thread saw the same barrier, so ok is uniform unless a wait
        // timed out on some threads only; make it uniform before the next copy
        ok = __syncthreads_and(ok ? 1 : 0) != 0;
    }
    if (!ok) {
        if (threadIdx.x == 0 && err) atomicExch(err, 1);
        umma_wait(bar_a, phase ^ 1u);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < UMMA_N; c0 += 8) {
            uint32_t v[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(lane_addr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < M)
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int n = n0 + c0 + j;
                    if (n < N) C[(size_t)row * ldc + n] = __uint_as_float(v[j]);
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UMMA_TMEM_COLS)
                     : "memory");
}

}  // namespace pimd
