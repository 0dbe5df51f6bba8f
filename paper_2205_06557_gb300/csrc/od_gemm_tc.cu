// BF16 matrix products of the warm-start network on the fifth-generation tensor cores:
// C[M][N] = A[M][K] B[N][K]^T (+ bias[N]) (relu), FP32 accumulation in tensor memory.
//
// One CTA of 128 threads computes a 128 x NT tile of C (NT <= 256, a multiple of 16 that
// divides N).  K is consumed in chunks of 32 (64 bytes of every row) through a ring of four
// shared-memory stages: the CTA's threads copy chunk c + 2 in with cp.async while the tensor
// cores multiply chunk c, so two chunks' copies are in flight behind the products.  Operands
// sit in shared memory in the canonical K-major layout without swizzling: 8-row x 16-byte
// core matrices, the 4 core matrices of a chunk's 8-row group side by side (128 bytes apart
// along K), the row groups 512 bytes apart.  One elected thread issues tcgen05.mma
// (M = 128, N = NT, K = 16, two per chunk) and commits each chunk's products to that stage's
// mbarrier, which the copy into the stage four chunks later waits for.  The accumulator
// lives in tensor memory (one lane per row of the tile, NT columns); the epilogue reads it
// with tcgen05.ld (warp w: rows 32w .. 32w + 31, 16 columns at a time), adds the bias,
// applies the relu and stages each 32 x 16 block in shared memory, so that the stores to C
// and to its BF16 copy write 64 contiguous bytes of a row per four lanes instead of one
// row per lane.
//
// Every wait on an mbarrier is bounded: a wait that runs out sets bit 1 of *err, stops
// the CTA's further products and still frees its tensor memory before returning.
#include <cuda_bf16.h>

#include <cstdint>

#include "od_internal.h"

namespace od {
namespace tc {

constexpr int BT = 128;                    // threads per CTA (four warps: 128 TMEM lanes)
constexpr int TM = 128;                    // tile rows
constexpr int TK = 32;                     // K per chunk (64 bytes of a BF16 row)
constexpr int STAGES = 4;                  // chunks in the shared-memory ring
constexpr int AHEAD = 2;                   // chunks copied ahead of the one multiplied
constexpr int NT_MAX = 256;                // widest tile (one MMA instruction's N)
constexpr int A_BYTES = TM * TK * 2;       // 8 KB
constexpr int B_BYTES = NT_MAX * TK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t SBO = 8 * TK * 2;       // bytes between 8-row groups (512)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 64;  // stages, alignment, barriers
constexpr int EPI_LD = 20;                 // staged epilogue row stride (floats; 80 B)
constexpr long long WAIT_LIMIT = 1ll << 22;  // polls of an mbarrier before giving up
static_assert(4 * 32 * EPI_LD * 4 <= STAGES * STAGE_BYTES, "epilogue staging fits the stages");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K-direction core-matrix) and stride
// (8-row-group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // version
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t instr_desc(int m, int n)
{
    return (1u << 4)                        // D format: F32
           | (1u << 7)                      // A format: BF16
           | (1u << 10)                     // B format: BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(m >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with this parity to complete; false if it did not
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity)
{
    for (long long it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid)
{
    const int n = valid ? 16 : 0;  // zero-fill when the row is outside the matrix
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

// copy a rows x 32 BF16 chunk (rows from r0, K from k0) into the core-matrix layout:
// thread t writes the 16 bytes at offset 16 t of the stage, i.e. row group t / 32, core
// matrix (t / 8) % 4 along K, row t % 8 within it
__device__ __forceinline__ void load_chunk(uint32_t dst, const __nv_bfloat16* __restrict__ src, int rows, int r0,
                                           int nrows, int K, int k0)
{
    const int n16 = rows * (TK / 8);
    for (int t = threadIdx.x; t < n16; t += BT) {
        const int rg = t >> 5, kg = (t >> 3) & 3, r = t & 7;
        const int row = r0 + rg * 8 + r, k = k0 + kg * 8;
        const bool valid = row < nrows && k < K;
        const __nv_bfloat16* p = valid ? src + (long long)row * K + k : src;
        cp_async16(dst + 16u * (uint32_t)t, p, valid);
    }
}

__global__ void __launch_bounds__(BT) k_gemm_tc(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                                                const float* __restrict__ bias, float* __restrict__ C,
                                                __nv_bfloat16* __restrict__ Cb, int M, int N, int K, int NT, int relu,
                                                int* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = (uint64_t*)(smem + STAGES * STAGE_BYTES);  // one barrier per stage
    uint32_t* tmem_slot = (uint32_t*)(bar + STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * NT;
    const uint32_t ncols = NT <= 32 ? 32u : NT <= 64 ? 64u : NT <= 128 ? 128u : 256u;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const uint32_t idesc = instr_desc(TM, NT);
    const int nchunks = (K + TK - 1) / TK;
    auto stage_a = [&](int c) { return smem_u32(smem + (c % STAGES) * STAGE_BYTES); };
    auto copy = [&](int c) {
        if (c < nchunks) {
            load_chunk(stage_a(c), A, TM, m0, M, K, c * TK);
            load_chunk(stage_a(c) + A_BYTES, B, NT, n0, N, K, c * TK);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");  // (empty past the last chunk)
    };
    unsigned phase[STAGES] = {0u, 0u, 0u, 0u};
    bool failed = false;
    for (int c = 0; c < AHEAD; ++c) copy(c);
    for (int c = 0; c < nchunks; ++c) {
        // the stage of chunk c + AHEAD was last read by the products of chunk c + AHEAD - STAGES
        const int cn = c + AHEAD, cold = cn - STAGES;
        if (cn < nchunks && cold >= 0) {
            const int st = cold % STAGES;
            const bool ok = mbar_wait(&bar[st], phase[st]);
            phase[st] ^= 1u;
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
        }
        copy(cn);
        // every group but the AHEAD newest is complete: chunk c has landed
        asm volatile("cp.async.wait_group %0;" ::"n"(AHEAD) : "memory");
        // make the copies visible to the tensor cores (the async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = stage_a(c), sb = sa + A_BYTES;
            const int ksteps = min(TK, K - c * TK) / 16;
            for (int kk = 0; kk < ksteps; ++kk) {
                // K = 16 per instruction: two core matrices along K, 256 bytes further on
                const uint64_t da = smem_desc(sa + 256u * kk, 128u, SBO);
                const uint64_t db = smem_desc(sb + 256u * kk, 128u, SBO);
                const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[c % STAGES]))
                         : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (!failed) {
        // the commits of the last STAGES chunks, oldest first (the loop waited for every
        // earlier one), so that no barrier still has an arrival pending when the CTA ends;
        // the last covers every product
        bool ok = true;
        for (int c = max(0, nchunks - STAGES); c < nchunks; ++c) {
            const int st = c % STAGES;
            ok = ok && mbar_wait(&bar[st], phase[st]);
            phase[st] ^= 1u;
        }
        if (__syncthreads_or(!ok)) failed = true;
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(err, 2);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the stages are free: warp w stages its 32 x 16 blocks in its own 2.5 KB
        float* stg = (float*)smem + warp * 32 * EPI_LD;
        const int rb = m0 + warp * 32;  // the warp's first row
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float o[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float x = __uint_as_float(v[e]);
                if (bias) x += __ldg(bias + n0 + c0 + e);
                if (relu) x = fmaxf(x, 0.f);
                o[e] = x;
            }
            // lane = row of the block: four 16-byte writes into its staged row
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *(float4*)(stg + lane * EPI_LD + 4 * q) = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
            __syncwarp();
            // lanes l and l + 8k (k = 0..3) write the four 16-byte quarters of row l % 8 (+ 8 it)
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int r = it * 8 + (lane & 7), q = lane >> 3;
                const float4 x = *(const float4*)(stg + r * EPI_LD + 4 * q);
                if (rb + r < M) {
                    const long long off = (long long)(rb + r) * N + n0 + c0 + 4 * q;
                    *(float4*)(C + off) = x;
                    if (Cb) {
                        __nv_bfloat162 h[2] = {__floats2bfloat162_rn(x.x, x.y), __floats2bfloat162_rn(x.z, x.w)};
                        *(uint2*)(Cb + off) = *(const uint2*)h;
                    }
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace tc
}  // namespace od

namespace od {

// widest tile width (a multiple of 16, at most 256) that divides N
int gemm_tc_tile(int N)
{
    for (int nt = 256; nt >= 16; nt -= 16)
        if (N % nt == 0) return nt;
    return 0;
}

int launch_gemm_tc(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C, __nv_bfloat16* Cb,
                   int M, int N, int K, int relu, int* err, cudaStream_t s)
{
    const int nt = gemm_tc_tile(N);
    if (M < 1 || K < 16 || K % 16 || nt == 0) return (int)cudaErrorInvalidValue;
    // (per function and device: set on every call, it costs no device work)
    const cudaError_t e =
        cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    const dim3 grid((M + tc::TM - 1) / tc::TM, N / nt);
    tc::k_gemm_tc<<<grid, tc::BT, tc::SMEM_BYTES, s>>>(A, B, bias, C, Cb, M, N, K, nt, relu, err);
    return (int)cudaGetLastError();
}

}  // namespace od
