// BF16 matrix products of the warm-start network on the fifth-generation tensor cores:
// C[M][N] = A[M][K] B[N][K]^T (+ bias[N]) (relu), FP32 accumulation in tensor memory.
//
// One CTA of 128 threads computes a 128 x NT tile of C (NT <= 128, a multiple of 16 that
// divides N; two CTAs per SM; the N tiles of a row block launch next to each other).  K is
// consumed in chunks of 64 (128 bytes of every row) through a ring of three shared-memory
// stages filled by the tensor memory accelerator (TMA).  One thread runs the pipeline: per
// chunk, a TMA load of the A tile (128 x 64) and of the B tile (NT x 64) into a stage, both
// completing on the stage's "full" mbarrier by their byte count; once a chunk has landed,
// its four tcgen05.mma (M = 128, N = NT, K = 16), committed to the stage's "empty" mbarrier,
// which the load of the chunk three later into that stage waits for.  Two chunks' loads
// are in flight behind the products.  The tiles arrive in the 128-byte swizzled layout (row
// r of a tile at 128 r bytes, its 16-byte pieces permuted by r mod 8) that the shared-memory
// descriptors name (SWIZZLE_128B, 1,024 bytes between 8-row groups, K steps of 32 bytes
// within the swizzle span); rows past M and columns past K are zero-filled by the loads.
// After the last chunk the four warps read the accumulator with tcgen05.ld (warp w: rows
// 32w .. 32w + 31, 32 columns at a time), add the bias, apply the relu and stage each
// 32 x 32 block in shared memory, so that the stores of C and of its BF16 copy write 128
// contiguous bytes of a row per eight lanes.
//
// Every wait on an mbarrier is bounded: a wait that runs out sets bit 1 of *err, stops
// the CTA's further products and still frees its tensor memory before returning.
#include <cuda.h>  // CUtensorMap and the encoder's types; the encoder itself is fetched
                   // through the runtime's entry-point query (no link to libcuda)
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "od_internal.h"

namespace od {
namespace tc {

constexpr int BT = 128;                    // threads per CTA (four warps: 128 TMEM lanes)
constexpr int TM = 128;                    // tile rows
constexpr int TK = 64;                     // K per chunk (128 bytes of a BF16 row: one swizzle span)
constexpr int STAGES = 3;                  // chunks in the shared-memory ring
constexpr int NT_MAX = 128;                // widest tile
constexpr int A_BYTES = TM * TK * 2;       // 16 KB
constexpr int B_BYTES = NT_MAX * TK * 2;   // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t SBO = 8 * TK * 2;       // bytes between 8-row groups (1,024)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 128;  // stages, alignment, barriers
constexpr int EPI_LD = 36;                 // staged epilogue row stride (floats; 144 B)
constexpr long long WAIT_LIMIT = 1ll << 22;  // polls of an mbarrier before giving up
static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "swizzled tiles start on 1,024-byte boundaries");
static_assert(4 * 32 * EPI_LD * 4 <= STAGES * STAGE_BYTES, "epilogue staging fits the stages");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a K-major tile in the 128-byte swizzled layout:
// start address, leading byte offset 16 (unused for this layout), stride byte offset
// 1,024 (8 rows of 128 bytes), descriptor version 1, layout type 2 (SWIZZLE_128B)
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
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

// the A and B tiles of chunk c into stage c % STAGES, completing on that stage's full barrier
__device__ __forceinline__ void load_chunk(const CUtensorMap* tmA, const CUtensorMap* tmB, uint8_t* smem,
                                           uint64_t* full, int c, int m0, int n0, uint32_t bytes)
{
    const int st = c % STAGES;
    const uint32_t sa = smem_u32(smem + st * STAGE_BYTES), sb = sa + A_BYTES, bar = smem_u32(&full[st]);
    const int k0 = c * TK;  // innermost coordinate: a multiple of 64 elements (128 bytes)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            sa),
        "l"((uint64_t)tmA), "r"(k0), "r"(m0), "r"(bar)
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            sb),
        "l"((uint64_t)tmB), "r"(k0), "r"(n0), "r"(bar)
        : "memory");
}

// tcgen05.ld of W = 16 or 32 consecutive accumulator columns of the warp's 32 lanes (rows),
// issued without waiting; tmem_wait(v) waits for every load the thread issued and names v as
// its operands, so that no use of v moves before it
template <int W>
__device__ __forceinline__ void tmem_issue(uint32_t taddr, uint32_t (&v)[W]);

template <>
__device__ __forceinline__ void tmem_issue<16>(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_issue<32>(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

template <int W>
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[W])
{
#pragma unroll
    for (int e = 0; e < W; e += 16)
        asm volatile("" : "+r"(v[e]), "+r"(v[e + 1]), "+r"(v[e + 2]), "+r"(v[e + 3]), "+r"(v[e + 4]), "+r"(v[e + 5]),
                     "+r"(v[e + 6]), "+r"(v[e + 7]), "+r"(v[e + 8]), "+r"(v[e + 9]), "+r"(v[e + 10]), "+r"(v[e + 11]),
                     "+r"(v[e + 12]), "+r"(v[e + 13]), "+r"(v[e + 14]), "+r"(v[e + 15])::"memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < W; e += 16)
        asm volatile("" : "+r"(v[e]), "+r"(v[e + 1]), "+r"(v[e + 2]), "+r"(v[e + 3]), "+r"(v[e + 4]), "+r"(v[e + 5]),
                     "+r"(v[e + 6]), "+r"(v[e + 7]), "+r"(v[e + 8]), "+r"(v[e + 9]), "+r"(v[e + 10]), "+r"(v[e + 11]),
                     "+r"(v[e + 12]), "+r"(v[e + 13]), "+r"(v[e + 14]), "+r"(v[e + 15])::"memory");
}

// One 32 x W block of the warp's rows (W = 16 or 32 columns from column col of C): bias, relu,
// then staged in shared memory (lane = row, W/4 16-byte writes; rows EPI_LD floats apart, so
// each 8-lane phase hits distinct banks) and stored with W/4 lanes per row, 128 (W = 32) or 64
// (W = 16) contiguous bytes of a row per instruction's row.
template <int W>
__device__ __forceinline__ void epilogue_block(const uint32_t (&v)[W], float* stg, int lane, int rb, int M, int N,
                                               int col, const float* __restrict__ bias, int relu,
                                               float* __restrict__ C, __nv_bfloat16* __restrict__ Cb)
{
    constexpr int QR = W / 4;     // 16-byte pieces per row
    constexpr int RPI = 32 / QR;  // rows per store instruction
    float o[W];
#pragma unroll
    for (int q = 0; q < QR; ++q) {
        // the bias in 16-byte loads (col is a multiple of 16, the bias 16-byte aligned)
        const float4 b4 = bias ? __ldg((const float4*)(bias + col) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float bq[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float x = __uint_as_float(v[4 * q + e]) + bq[e];
            if (relu) x = fmaxf(x, 0.f);
            o[4 * q + e] = x;
        }
    }
#pragma unroll
    for (int q = 0; q < QR; ++q)
        *(float4*)(stg + lane * EPI_LD + 4 * q) = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (int it = 0; it < QR; ++it) {
        // W = 32: lanes 8k .. 8k + 7 write row 4 it + k; W = 16: lanes l, l + 8, l + 16, l + 24
        // write the four pieces of row 8 it + l % 8
        const int r = W == 32 ? it * RPI + (lane >> 3) : it * RPI + (lane & 7);
        const int q = W == 32 ? (lane & 7) : (lane >> 3);
        const float4 x = *(const float4*)(stg + r * EPI_LD + 4 * q);
        if (rb + r < M) {
            const long long off = (long long)(rb + r) * N + col + 4 * q;
            *(float4*)(C + off) = x;
            if (Cb) {
                __nv_bfloat162 h[2] = {__floats2bfloat162_rn(x.x, x.y), __floats2bfloat162_rn(x.z, x.w)};
                *(uint2*)(Cb + off) = *(const uint2*)h;
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(BT) k_gemm_tc(const __grid_constant__ CUtensorMap tmA,
                                                const __grid_constant__ CUtensorMap tmB, const float* __restrict__ bias,
                                                float* __restrict__ C, __nv_bfloat16* __restrict__ Cb, int M, int N,
                                                int K, int NT, int relu, int* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);  // loads landed, per stage
    uint64_t* empty = full + STAGES;                             // products done reading, per stage
    uint32_t* tmem_slot = (uint32_t*)(empty + STAGES);
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the N tiles of one row block are neighbours in launch order, so they run together and
    // the second reads the A tile from L2
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * NT;
    const uint32_t ncols = NT <= 32 ? 32u : NT <= 64 ? 64u : 128u;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
        s_fail = 0;
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

    if (threadIdx.x == 0) {
        // the pipeline, in one thread: products of chunk c, then the load of chunk c + 2 into
        // the stage that the products of chunk c - 1 read
        const uint32_t idesc = instr_desc(TM, NT);
        const uint32_t bytes = (uint32_t)(A_BYTES + NT * TK * 2);  // the two boxes (zero-filled parts count)
        const int nchunks = (K + TK - 1) / TK;
        unsigned ph_full[STAGES] = {}, ph_empty[STAGES] = {};
        bool ok = true;
        for (int c = 0; c < STAGES - 1 && c < nchunks; ++c) load_chunk(&tmA, &tmB, smem, full, c, m0, n0, bytes);
        int waited_to = -1;  // the products of chunks up to this one are known to be done
        for (int c = 0; c < nchunks && ok; ++c) {
            const int st = c % STAGES;
            ok = mbar_wait(&full[st], ph_full[st]);
            ph_full[st] ^= 1u;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + st * STAGE_BYTES), sb = sa + A_BYTES;
            const int ksteps = min(TK, K - c * TK) / 16;
            for (int kk = 0; kk < ksteps; ++kk) {
                // K = 16 per instruction: 32 bytes further along the 128-byte swizzle span
                const uint64_t da = smem_desc_sw128(sa + 32u * kk);
                const uint64_t db = smem_desc_sw128(sb + 32u * kk);
                const uint32_t accum = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[st]))
                         : "memory");
            const int cn = c + STAGES - 1;
            if (cn < nchunks) {
                if (cn >= STAGES) {
                    // chunk cn - STAGES = c - 1 last read this stage
                    const int so = (cn - STAGES) % STAGES;
                    ok = mbar_wait(&empty[so], ph_empty[so]);
                    ph_empty[so] ^= 1u;
                    waited_to = cn - STAGES;
                    if (!ok) break;
                }
                load_chunk(&tmA, &tmB, smem, full, cn, m0, n0, bytes);
            }
        }
        // the commits not waited for yet, oldest first: then every product is done and no
        // barrier has an arrival pending when the CTA ends
        for (int c = waited_to + 1; c < nchunks && ok; ++c) {
            const int st = c % STAGES;
            ok = mbar_wait(&empty[st], ph_empty[st]);
            ph_empty[st] ^= 1u;
        }
        if (!ok) {
            s_fail = 1;
            atomicOr(err, 2);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (!s_fail) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the stages are free: warp w stages its blocks in its own 4.5 KB
        float* stg = (float*)smem + warp * 32 * EPI_LD;
        const int rb = m0 + warp * 32;  // the warp's first row
        const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
        const int n32 = NT / 32;
        if (n32 > 0) {
            // the next block's columns are read from tensor memory while this block is stored
            uint32_t va[32], vb[32];
            tmem_issue<32>(tw, va);
            tmem_wait<32>(va);
            for (int b = 0; b < n32; b += 2) {
                if (b + 1 < n32) tmem_issue<32>(tw + (uint32_t)(32 * (b + 1)), vb);
                epilogue_block<32>(va, stg, lane, rb, M, N, n0 + 32 * b, bias, relu, C, Cb);
                if (b + 1 >= n32) break;
                tmem_wait<32>(vb);
                if (b + 2 < n32) tmem_issue<32>(tw + (uint32_t)(32 * (b + 2)), va);
                epilogue_block<32>(vb, stg, lane, rb, M, N, n0 + 32 * (b + 1), bias, relu, C, Cb);
                if (b + 2 < n32) tmem_wait<32>(va);
            }
        }
        if (NT % 32) {
            uint32_t v16[16];
            tmem_issue<16>(tw + (uint32_t)(32 * n32), v16);
            tmem_wait<16>(v16);
            epilogue_block<16>(v16, stg, lane, rb, M, N, n0 + 32 * n32, bias, relu, C, Cb);
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

// widest tile width (a multiple of 16, at most 128) that divides N
int gemm_tc_tile(int N)
{
    for (int nt = tc::NT_MAX; nt >= 16; nt -= 16)
        if (N % nt == 0) return nt;
    return 0;
}

namespace {

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
        cudaGetLastError();
    });
    return fn;
}

// a rows x K BF16 row-major matrix, read in boxes of box_rows x 64 with the 128-byte swizzle;
// reads past the matrix return zeros
bool encode(CUtensorMap* tm, const __nv_bfloat16* base, int rows, int K, int box_rows)
{
    const EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)tc::TK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int launch_gemm_tc(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C, __nv_bfloat16* Cb,
                   int M, int N, int K, int relu, int* err, cudaStream_t s)
{
    const int nt = gemm_tc_tile(N);
    if (M < 1 || K < 16 || K % 16 || nt == 0) return (int)cudaErrorInvalidValue;
    // TMA: 16-byte aligned bases (row strides are multiples of 16 bytes since K % 16 == 0);
    // the epilogue's 16-byte stores and bias loads: 16-byte aligned C, Cb and bias
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C | (uintptr_t)Cb | (uintptr_t)bias) & 15)
        return (int)cudaErrorMisalignedAddress;
    alignas(64) CUtensorMap tmA, tmB;
    if (!encode(&tmA, A, M, K, tc::TM) || !encode(&tmB, B, N, K, nt)) return (int)cudaErrorInvalidValue;
    // (per function and device: set on every call, it costs no device work)
    const cudaError_t e =
        cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    if (e != cudaSuccess) return (int)e;
    const dim3 grid(N / nt, (M + tc::TM - 1) / tc::TM);
    if (grid.y > 65535u) return (int)cudaErrorInvalidValue;
    tc::k_gemm_tc<<<grid, tc::BT, tc::SMEM_BYTES, s>>>(tmA, tmB, bias, C, Cb, M, N, K, nt, relu, err);
    return (int)cudaGetLastError();
}

}  // namespace od
