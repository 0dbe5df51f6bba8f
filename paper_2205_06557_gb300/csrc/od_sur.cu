// Learned warm start for the self-consistent grain charge: a small set-pooled MLP,
// trained on the GPU by the library's own forward, backward and Adam kernels.
//
// Network (per grain k of a sample, grains masked, at most 8 per sample):
//   x_k  = [global features (3), grain features (4)], padded to 16
//   h1_k = relu(W1 x_k + b1)            256
//   h2_k = relu(W2 h1_k + b2)           256
//   c    = mean over present grains of h2_k (set pooling)
//   h3_k = relu(W3 [h2_k, c] + b3)      256
//   h4_k = relu(W4 h3_k + b4)           256
//   y_k  = W5 h4_k + b5                 4 outputs (padded to 16)
// Weights are kept in FP32 (master copy for Adam) and used as BF16 in every matrix
// product (BF16 inputs, FP32 accumulation: tcgen05.mma tiles by default, od_gemm_tc.cu,
// or warp-level mma.sync m16n8k16 tiles, k_gemm_nt below);
// activations are rounded to BF16 where they enter a product.  The loss is the mean
// squared error over present grains and the four outputs.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "od_internal.h"

namespace od {
namespace sur {

constexpr int IN = 7, K0 = 16, H = 256, OUTR = 4, OUTP = 16, G = 8;

// ------------------------------------------------------------------ GEMM
// C[M][N] = A[M][K] * B[N][K]^T (+ bias[N]) (relu) in FP32, optional BF16 copy.
// A, B BF16 row-major; M, N, K multiples of 16.  One warp per 16x16 output tile,
// two m16n8k16 products per k-step of 16.
__device__ __forceinline__ unsigned ld2(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

__global__ void k_gemm_nt(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                          const float* __restrict__ bias, float* __restrict__ C, __nv_bfloat16* __restrict__ Cb,
                          int M, int N, int K, int relu)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int tiles_n = N / 16;
    if (warp >= (M / 16) * tiles_n) return;
    const int m0 = (warp / tiles_n) * 16, n0 = (warp % tiles_n) * 16;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int k0 = 0; k0 < K; k0 += 16) {
        const __nv_bfloat16* a_lo = A + (long long)(m0 + g) * K + k0 + 2 * t;
        const __nv_bfloat16* a_hi = A + (long long)(m0 + g + 8) * K + k0 + 2 * t;
        const unsigned a0 = ld2(a_lo), a1 = ld2(a_hi), a2 = ld2(a_lo + 8), a3 = ld2(a_hi + 8);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const __nv_bfloat16* bp = B + (long long)(n0 + 8 * s + g) * K + k0 + 2 * t;
            const unsigned b0 = ld2(bp), b1 = ld2(bp + 8);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(acc[s][0]), "+f"(acc[s][1]), "+f"(acc[s][2]), "+f"(acc[s][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = m0 + g + 8 * h;
            const int col = n0 + 8 * s + 2 * t;
            float v0 = acc[s][2 * h], v1 = acc[s][2 * h + 1];
            if (bias) {
                v0 += bias[col];
                v1 += bias[col + 1];
            }
            if (relu) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
            }
            C[(long long)row * N + col] = v0;
            C[(long long)row * N + col + 1] = v1;
            if (Cb) {
                Cb[(long long)row * N + col] = __float2bfloat16_rn(v0);
                Cb[(long long)row * N + col + 1] = __float2bfloat16_rn(v1);
            }
        }
}

// ---------------------------------------------------------------- helpers
__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// out[c][r] = in[r][c] (BF16), in is R x C
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out, int R, int C)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)R * C) return;
    const int r = (int)(i / C), c = (int)(i % C);
    out[(long long)c * R + r] = in[i];
}

// masked mean over the G grains of each sample: c[b][j] = sum_k m_bk h[bG+k][j] / n_b
__global__ void k_pool(const float* __restrict__ h, const float* __restrict__ mask, float* __restrict__ c, int Bn)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bn * H) return;
    const int b = i / H, j = i % H;
    float s = 0.f, n = 0.f;
    for (int k = 0; k < G; ++k) {
        const float m = mask[b * G + k];
        s += m * h[(long long)(b * G + k) * H + j];
        n += m;
    }
    c[i] = n > 0.f ? s / n : 0.f;
}

// X3[row] = [h2[row], c[sample]] as BF16
__global__ void k_concat(const __nv_bfloat16* __restrict__ h2b, const float* __restrict__ c,
                         __nv_bfloat16* __restrict__ x3, int M)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * 2 * H) return;
    const int row = (int)(i / (2 * H)), j = (int)(i % (2 * H));
    x3[i] = j < H ? h2b[(long long)row * H + j] : __float2bfloat16_rn(c[(row / G) * H + (j - H)]);
}

// dY = 2 (y - t) / count on present grains and real outputs; loss partial sums per row
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ tgt, const float* __restrict__ mask,
                       float* __restrict__ dy, float* __restrict__ row_loss, int M, float inv_count)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= M) return;
    const float m = mask[row];
    float l = 0.f;
    for (int o = 0; o < OUTP; ++o) {
        float d = 0.f;
        if (o < OUTR && m > 0.f) {
            const float e = y[row * OUTP + o] - tgt[row * OUTR + o];
            l += e * e;
            d = 2.f * e * inv_count;
        }
        dy[row * OUTP + o] = d;
    }
    row_loss[row] = l * inv_count;
}

// dZ = dA * (Z > 0) in place on dA (Z holds post-relu values: > 0 iff pre-activation > 0)
__global__ void k_relu_back(float* __restrict__ da, const float* __restrict__ a, __nv_bfloat16* __restrict__ dzb,
                            long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = a[i] > 0.f ? da[i] : 0.f;
    da[i] = v;
    dzb[i] = __float2bfloat16_rn(v);
}

// column sums of dZ [M][N] -> db[N] (fixed order per column)
__global__ void k_colsum(const float* __restrict__ dz, float* __restrict__ db, int M, int N)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int r = 0; r < M; ++r) s += dz[(long long)r * N + j];
    db[j] = s;
}

// split dX3 [M][2H]: dA2 = first half + pooled share of the second half
__global__ void k_unpool(const float* __restrict__ dx3, const float* __restrict__ mask, float* __restrict__ da2, int M)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)M * H) return;
    const int row = (int)(i / H), j = (int)(i % H);
    const int b = row / G;
    float n = 0.f, dc = 0.f;
    for (int k = 0; k < G; ++k) {
        const float m = mask[b * G + k];
        n += m;
        dc += m * dx3[(long long)(b * G + k) * 2 * H + H + j];
    }
    const float share = n > 0.f ? mask[row] * dc / n : 0.f;
    da2[i] = dx3[(long long)row * 2 * H + j] + share;
}

// Adam on FP32 master parameters, then the BF16 copy (and its transpose for weights)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, __nv_bfloat16* __restrict__ pbt, int rows, int cols, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
    if (pbt) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        pbt[(long long)c * rows + r] = __float2bfloat16_rn(pi);
    }
}

}  // namespace sur
}  // namespace od

using namespace od;
using namespace od::sur;

// ------------------------------------------------------------------- host
namespace {

struct Layer {
    int out, in;
    float *w = nullptr, *b = nullptr;        // FP32 master
    float *gw = nullptr, *gb = nullptr;      // gradients
    float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;  // Adam moments
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;  // BF16 copy [out][in] and transpose [in][out]
};

}  // namespace

struct od_sur {
    int maxB = 0;
    Layer L[5];
    // activations, M = maxB * G rows
    __nv_bfloat16 *x0b, *h1b, *h2b, *x3b, *h3b, *h4b, *dyb, *dzb, *tA, *tB;
    float *h1, *h2, *c, *h3, *h4, *y, *dy, *dx, *dx3, *da, *rowl, *mask, *tgt, *xin;
    cudaStream_t stream = nullptr;
    long long adam_t = 0;
    int engine = OD_GEMM_TCGEN05;
    int* d_err = nullptr;  // tensor-core wait timeouts (bit 1)
    std::string err;
};

namespace {

thread_local std::string g_sur_error;

int sfail(od_sur* s, int code, const std::string& msg)
{
    if (s) s->err = msg;
    else g_sur_error = msg;
    return code;
}

#define SCK(s, call)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return sfail(s, OD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

inline int blocks(long long n, int bt = 256) { return (int)((n + bt - 1) / bt); }

}  // namespace

namespace od {
int launch_gemm_tc(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C, __nv_bfloat16* Cb,
                   int M, int N, int K, int relu, int* err, cudaStream_t s);

int gemm_bf16(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C, __nv_bfloat16* Cb, int M,
              int N, int K, int relu, int engine, int* err, cudaStream_t stream)
{
    if (engine == OD_GEMM_TCGEN05) return launch_gemm_tc(A, B, bias, C, Cb, M, N, K, relu, err, stream);
    const long long warps = (long long)(M / 16) * (N / 16);
    k_gemm_nt<<<blocks(warps * 32, 128), 128, 0, stream>>>(A, B, bias, C, Cb, M, N, K, relu);
    return (int)cudaGetLastError();
}
}  // namespace od

namespace {

int gemm(od_sur* s, const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* C, __nv_bfloat16* Cb, int M,
         int N, int K, int relu)
{
    const int e = gemm_bf16(A, B, bias, C, Cb, M, N, K, relu, s->engine, s->d_err, s->stream);
    return e == 0 ? OD_OK : sfail(s, OD_ECUDA, std::string("gemm launch failed: ") + cudaGetErrorString((cudaError_t)e));
}

// tensor-core waits that gave up since the last check (read after a synchronisation)
int check_engine(od_sur* s)
{
    int e = 0;
    SCK(s, cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SCK(s, cudaStreamSynchronize(s->stream));
    if (e) {
        SCK(s, cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
        return sfail(s, OD_ETIMEOUT, "a tensor-core product's wait gave up");
    }
    return OD_OK;
}

void free_sur(od_sur* s)
{
    for (auto& l : s->L) {
        cudaFree(l.w), cudaFree(l.b), cudaFree(l.gw), cudaFree(l.gb), cudaFree(l.mw), cudaFree(l.vw), cudaFree(l.mb),
            cudaFree(l.vb), cudaFree(l.wb), cudaFree(l.wt);
    }
    void* bufs[] = {s->x0b, s->h1b, s->h2b, s->x3b, s->h3b, s->h4b, s->dyb, s->dzb, s->tA, s->tB, s->h1, s->h2,
                    s->c, s->h3, s->h4, s->y, s->dy, s->dx, s->dx3, s->da, s->rowl, s->mask, s->tgt, s->xin};
    for (void* p : bufs) cudaFree(p);
    cudaFree(s->d_err);
}

// refresh the BF16 copies of every layer from the FP32 masters
int refresh_bf16(od_sur* s)
{
    for (auto& l : s->L) {
        const long long n = (long long)l.out * l.in;
        k_to_bf16<<<blocks(n), 256, 0, s->stream>>>(l.w, l.wb, n);
        k_transpose<<<blocks(n), 256, 0, s->stream>>>(l.wb, l.wt, l.out, l.in);
    }
    return cudaGetLastError() == cudaSuccess ? OD_OK : sfail(s, OD_ECUDA, "weight refresh failed");
}

// inputs: xin [B][G][IN] FP32 (host layout copied), mask [B][G]
int forward(od_sur* s, int Bn)
{
    const int M = Bn * G;
    // x0 padded to K0 columns
    {
        std::vector<float> dummy;  // padding is done on the host when uploading
    }
    int rc;
    if ((rc = gemm(s, s->x0b, s->L[0].wb, s->L[0].b, s->h1, s->h1b, M, H, K0, 1))) return rc;
    if ((rc = gemm(s, s->h1b, s->L[1].wb, s->L[1].b, s->h2, s->h2b, M, H, H, 1))) return rc;
    k_pool<<<blocks((long long)Bn * H), 256, 0, s->stream>>>(s->h2, s->mask, s->c, Bn);
    k_concat<<<blocks((long long)M * 2 * H), 256, 0, s->stream>>>(s->h2b, s->c, s->x3b, M);
    if ((rc = gemm(s, s->x3b, s->L[2].wb, s->L[2].b, s->h3, s->h3b, M, H, 2 * H, 1))) return rc;
    if ((rc = gemm(s, s->h3b, s->L[3].wb, s->L[3].b, s->h4, s->h4b, M, H, H, 1))) return rc;
    if ((rc = gemm(s, s->h4b, s->L[4].wb, s->L[4].b, s->y, nullptr, M, OUTP, H, 0))) return rc;
    return OD_OK;
}

// dW = dZ^T X over the M rows (NT product of the transposes), db = column sums
int weight_grad(od_sur* s, Layer& l, const float* dz, const __nv_bfloat16* dzb, const __nv_bfloat16* xb, int M)
{
    k_transpose<<<blocks((long long)M * l.out), 256, 0, s->stream>>>(dzb, s->tA, M, l.out);
    k_transpose<<<blocks((long long)M * l.in), 256, 0, s->stream>>>(xb, s->tB, M, l.in);
    int rc = gemm(s, s->tA, s->tB, nullptr, l.gw, nullptr, l.out, l.in, M, 0);
    if (rc) return rc;
    k_colsum<<<blocks(l.out), 256, 0, s->stream>>>(dz, l.gb, M, l.out);
    return OD_OK;
}

int backward(od_sur* s, int Bn)
{
    const int M = Bn * G;
    int rc;
    // output layer: dy (FP32) -> BF16
    k_to_bf16<<<blocks((long long)M * OUTP), 256, 0, s->stream>>>(s->dy, s->dyb, (long long)M * OUTP);
    if ((rc = weight_grad(s, s->L[4], s->dy, s->dyb, s->h4b, M))) return rc;
    // dh4 = dy W5  (B = W5^T [H][OUTP])
    if ((rc = gemm(s, s->dyb, s->L[4].wt, nullptr, s->da, nullptr, M, H, OUTP, 0))) return rc;
    k_relu_back<<<blocks((long long)M * H), 256, 0, s->stream>>>(s->da, s->h4, s->dzb, (long long)M * H);
    if ((rc = weight_grad(s, s->L[3], s->da, s->dzb, s->h3b, M))) return rc;
    if ((rc = gemm(s, s->dzb, s->L[3].wt, nullptr, s->da, nullptr, M, H, H, 0))) return rc;
    k_relu_back<<<blocks((long long)M * H), 256, 0, s->stream>>>(s->da, s->h3, s->dzb, (long long)M * H);
    if ((rc = weight_grad(s, s->L[2], s->da, s->dzb, s->x3b, M))) return rc;
    if ((rc = gemm(s, s->dzb, s->L[2].wt, nullptr, s->dx3, nullptr, M, 2 * H, H, 0))) return rc;
    k_unpool<<<blocks((long long)M * H), 256, 0, s->stream>>>(s->dx3, s->mask, s->da, M);
    k_relu_back<<<blocks((long long)M * H), 256, 0, s->stream>>>(s->da, s->h2, s->dzb, (long long)M * H);
    if ((rc = weight_grad(s, s->L[1], s->da, s->dzb, s->h1b, M))) return rc;
    if ((rc = gemm(s, s->dzb, s->L[1].wt, nullptr, s->da, nullptr, M, H, H, 0))) return rc;
    k_relu_back<<<blocks((long long)M * H), 256, 0, s->stream>>>(s->da, s->h1, s->dzb, (long long)M * H);
    if ((rc = weight_grad(s, s->L[0], s->da, s->dzb, s->x0b, M))) return rc;
    return cudaGetLastError() == cudaSuccess ? OD_OK : sfail(s, OD_ECUDA, "backward launch failed");
}

int upload_batch(od_sur* s, const float* x, const float* mask, const float* tgt, int Bn)
{
    const int M = Bn * G;
    std::vector<float> xp((size_t)M * K0, 0.f);
    for (int r = 0; r < M; ++r)
        for (int j = 0; j < IN; ++j) xp[(size_t)r * K0 + j] = x[(size_t)r * IN + j];
    SCK(s, cudaMemcpyAsync(s->xin, xp.data(), sizeof(float) * xp.size(), cudaMemcpyHostToDevice, s->stream));
    k_to_bf16<<<blocks((long long)M * K0), 256, 0, s->stream>>>(s->xin, s->x0b, (long long)M * K0);
    SCK(s, cudaMemcpyAsync(s->mask, mask, sizeof(float) * M, cudaMemcpyHostToDevice, s->stream));
    if (tgt) SCK(s, cudaMemcpyAsync(s->tgt, tgt, sizeof(float) * M * OUTR, cudaMemcpyHostToDevice, s->stream));
    return OD_OK;
}

int loss_and_grad(od_sur* s, int Bn, const float* mask_host, double* loss)
{
    const int M = Bn * G;
    double cnt = 0.0;
    for (int r = 0; r < M; ++r) cnt += mask_host[r] > 0.f ? 1.0 : 0.0;
    const float inv = cnt > 0 ? (float)(1.0 / (cnt * OUTR)) : 0.f;
    int rc = forward(s, Bn);
    if (rc) return rc;
    k_loss<<<blocks(M), 256, 0, s->stream>>>(s->y, s->tgt, s->mask, s->dy, s->rowl, M, inv);
    if ((rc = backward(s, Bn))) return rc;
    if (loss) {
        std::vector<float> rl(M);
        SCK(s, cudaMemcpyAsync(rl.data(), s->rowl, sizeof(float) * M, cudaMemcpyDeviceToHost, s->stream));
        SCK(s, cudaStreamSynchronize(s->stream));
        double l = 0.0;
        for (float v : rl) l += v;
        *loss = l;
    }
    return OD_OK;
}

}  // namespace

extern "C" {

int od_sur_create(int max_batch, uint64_t seed, void* stream, od_sur** out)
{
    if (!out || max_batch < 1 || max_batch > (1 << 16)) return sfail(nullptr, OD_EINVAL, "bad surrogate arguments");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return sfail(nullptr, OD_ENODEV, "no CUDA device");
    od_sur* s = new od_sur();
    std::memset((void*)&s->x0b, 0, sizeof(void*) * 24);
    s->maxB = (max_batch + 1) / 2 * 2;  // M = 8 B rows must be a multiple of 16
    s->stream = (cudaStream_t)stream;
    const int dims[5][2] = {{H, K0}, {H, H}, {H, 2 * H}, {H, H}, {OUTP, H}};
    // He-uniform initial weights from a seeded host generator (splitmix64), zero biases
    unsigned long long st = seed * 0x9E3779B97F4A7C15ull + 12345ull;
    auto next = [&st]() {
        unsigned long long z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    bool ok = true;
    for (int li = 0; li < 5 && ok; ++li) {
        Layer& l = s->L[li];
        l.out = dims[li][0];
        l.in = dims[li][1];
        const size_t nw = (size_t)l.out * l.in;
        const int fan_in = li == 0 ? IN : l.in;
        const double bound = std::sqrt(6.0 / fan_in) * (li == 4 ? 0.1 : 1.0);
        std::vector<float> w(nw, 0.f);
        for (int o = 0; o < l.out; ++o)
            for (int i = 0; i < l.in; ++i) {
                const bool live = (li != 0 || i < IN) && (li != 4 || o < OUTR);
                const double u = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
                w[(size_t)o * l.in + i] = live ? (float)((2.0 * u - 1.0) * bound) : 0.f;
            }
        ok = cudaMalloc(&l.w, sizeof(float) * nw) == cudaSuccess && cudaMalloc(&l.b, sizeof(float) * l.out) == cudaSuccess &&
             cudaMalloc(&l.gw, sizeof(float) * nw) == cudaSuccess && cudaMalloc(&l.gb, sizeof(float) * l.out) == cudaSuccess &&
             cudaMalloc(&l.mw, sizeof(float) * nw) == cudaSuccess && cudaMalloc(&l.vw, sizeof(float) * nw) == cudaSuccess &&
             cudaMalloc(&l.mb, sizeof(float) * l.out) == cudaSuccess && cudaMalloc(&l.vb, sizeof(float) * l.out) == cudaSuccess &&
             cudaMalloc(&l.wb, sizeof(__nv_bfloat16) * nw) == cudaSuccess &&
             cudaMalloc(&l.wt, sizeof(__nv_bfloat16) * nw) == cudaSuccess;
        if (!ok) break;
        cudaMemcpyAsync(l.w, w.data(), sizeof(float) * nw, cudaMemcpyHostToDevice, s->stream);
        cudaMemsetAsync(l.b, 0, sizeof(float) * l.out, s->stream);
        cudaMemsetAsync(l.mw, 0, sizeof(float) * nw, s->stream);
        cudaMemsetAsync(l.vw, 0, sizeof(float) * nw, s->stream);
        cudaMemsetAsync(l.mb, 0, sizeof(float) * l.out, s->stream);
        cudaMemsetAsync(l.vb, 0, sizeof(float) * l.out, s->stream);
    }
    const long long M = (long long)s->maxB * G;
    auto mb = [&](void** p, size_t bytes) { ok = ok && cudaMalloc(p, bytes) == cudaSuccess; };
    mb((void**)&s->x0b, 2 * M * K0);
    mb((void**)&s->h1b, 2 * M * H);
    mb((void**)&s->h2b, 2 * M * H);
    mb((void**)&s->x3b, 2 * M * 2 * H);
    mb((void**)&s->h3b, 2 * M * H);
    mb((void**)&s->h4b, 2 * M * H);
    mb((void**)&s->dyb, 2 * M * OUTP);
    mb((void**)&s->dzb, 2 * M * H);
    mb((void**)&s->tA, 2 * M * 2 * H);
    mb((void**)&s->tB, 2 * M * 2 * H);
    mb((void**)&s->h1, 4 * M * H);
    mb((void**)&s->h2, 4 * M * H);
    mb((void**)&s->c, 4 * (long long)s->maxB * H);
    mb((void**)&s->h3, 4 * M * H);
    mb((void**)&s->h4, 4 * M * H);
    mb((void**)&s->y, 4 * M * OUTP);
    mb((void**)&s->dy, 4 * M * OUTP);
    mb((void**)&s->dx, 4 * M * H);
    mb((void**)&s->dx3, 4 * M * 2 * H);
    mb((void**)&s->da, 4 * M * 2 * H);
    mb((void**)&s->rowl, 4 * M);
    mb((void**)&s->mask, 4 * M);
    mb((void**)&s->tgt, 4 * M * OUTR);
    mb((void**)&s->xin, 4 * M * K0);
    mb((void**)&s->d_err, sizeof(int));
    if (ok) ok = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream) == cudaSuccess;
    if (!ok || refresh_bf16(s) != OD_OK || cudaStreamSynchronize(s->stream) != cudaSuccess) {
        g_sur_error = "surrogate allocation failed";
        free_sur(s);
        delete s;
        return OD_ENOMEM;
    }
    *out = s;
    return OD_OK;
}

void od_sur_destroy(od_sur* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    free_sur(s);
    delete s;
}

int od_sur_num_params(const od_sur* s)
{
    if (!s) return 0;
    int n = 0;
    for (const auto& l : s->L) n += l.out * l.in + l.out;
    return n;
}

// FP32 master parameters, layer by layer: W (out x in, row-major) then b (out)
int od_sur_get_params(od_sur* s, float* host)
{
    if (!s || !host) return sfail(s, OD_EINVAL, "bad argument");
    size_t off = 0;
    for (auto& l : s->L) {
        SCK(s, cudaMemcpyAsync(host + off, l.w, sizeof(float) * l.out * l.in, cudaMemcpyDeviceToHost, s->stream));
        off += (size_t)l.out * l.in;
        SCK(s, cudaMemcpyAsync(host + off, l.b, sizeof(float) * l.out, cudaMemcpyDeviceToHost, s->stream));
        off += l.out;
    }
    SCK(s, cudaStreamSynchronize(s->stream));
    return OD_OK;
}

int od_sur_set_params(od_sur* s, const float* host)
{
    if (!s || !host) return sfail(s, OD_EINVAL, "bad argument");
    size_t off = 0;
    for (auto& l : s->L) {
        SCK(s, cudaMemcpyAsync(l.w, host + off, sizeof(float) * l.out * l.in, cudaMemcpyHostToDevice, s->stream));
        off += (size_t)l.out * l.in;
        SCK(s, cudaMemcpyAsync(l.b, host + off, sizeof(float) * l.out, cudaMemcpyHostToDevice, s->stream));
        off += l.out;
    }
    int rc = refresh_bf16(s);
    if (rc) return rc;
    SCK(s, cudaStreamSynchronize(s->stream));
    return OD_OK;
}

// y[B][G][4] for inputs x[B][G][7] (host) and mask[B][G] (host)
int od_sur_forward(od_sur* s, const float* x, const float* mask, int Bn, float* y)
{
    if (!s || !x || !mask || !y || Bn < 1 || Bn > s->maxB) return sfail(s, OD_EINVAL, "bad forward arguments");
    const int Bp = (Bn + 1) / 2 * 2, M = Bp * G;
    std::vector<float> xs((size_t)M * IN, 0.f), ms(M, 0.f);
    std::memcpy(xs.data(), x, sizeof(float) * Bn * G * IN);
    std::memcpy(ms.data(), mask, sizeof(float) * Bn * G);
    int rc = upload_batch(s, xs.data(), ms.data(), nullptr, Bp);
    if (rc) return rc;
    if ((rc = forward(s, Bp))) return rc;
    std::vector<float> yy((size_t)M * OUTP);
    SCK(s, cudaMemcpyAsync(yy.data(), s->y, sizeof(float) * yy.size(), cudaMemcpyDeviceToHost, s->stream));
    if ((rc = check_engine(s))) return rc;
    for (int r = 0; r < Bn * G; ++r)
        for (int o = 0; o < OUTR; ++o) y[(size_t)r * OUTR + o] = yy[(size_t)r * OUTP + o];
    return OD_OK;
}

// loss and parameter gradients (layout of od_sur_get_params) without an update
int od_sur_gradients(od_sur* s, const float* x, const float* mask, const float* tgt, int Bn, double* loss, float* grads)
{
    if (!s || !x || !mask || !tgt || Bn < 1 || Bn > s->maxB) return sfail(s, OD_EINVAL, "bad gradient arguments");
    const int Bp = (Bn + 1) / 2 * 2, M = Bp * G;
    std::vector<float> xs((size_t)M * IN, 0.f), ms(M, 0.f), ts((size_t)M * OUTR, 0.f);
    std::memcpy(xs.data(), x, sizeof(float) * Bn * G * IN);
    std::memcpy(ms.data(), mask, sizeof(float) * Bn * G);
    std::memcpy(ts.data(), tgt, sizeof(float) * Bn * G * OUTR);
    int rc = upload_batch(s, xs.data(), ms.data(), ts.data(), Bp);
    if (rc) return rc;
    if ((rc = loss_and_grad(s, Bp, ms.data(), loss))) return rc;
    if (loss && (rc = check_engine(s))) return rc;
    if (grads) {
        size_t off = 0;
        for (auto& l : s->L) {
            SCK(s, cudaMemcpyAsync(grads + off, l.gw, sizeof(float) * l.out * l.in, cudaMemcpyDeviceToHost, s->stream));
            off += (size_t)l.out * l.in;
            SCK(s, cudaMemcpyAsync(grads + off, l.gb, sizeof(float) * l.out, cudaMemcpyDeviceToHost, s->stream));
            off += l.out;
        }
        if ((rc = check_engine(s))) return rc;
    }
    return OD_OK;
}

// one Adam step on a minibatch; returns the minibatch loss
int od_sur_train_step(od_sur* s, const float* x, const float* mask, const float* tgt, int Bn, float lr, double* loss)
{
    int rc = od_sur_gradients(s, x, mask, tgt, Bn, loss, nullptr);
    if (rc) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    s->adam_t += 1;
    const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
    for (auto& l : s->L) {
        const long long nw = (long long)l.out * l.in;
        k_adam<<<blocks(nw), 256, 0, s->stream>>>(l.w, l.gw, l.mw, l.vw, l.wb, l.wt, l.out, l.in, lr, b1, b2, eps, c1, c2);
        k_adam<<<blocks(l.out), 256, 0, s->stream>>>(l.b, l.gb, l.mb, l.vb, nullptr, nullptr, 1, l.out, lr, b1, b2, eps, c1,
                                                      c2);
    }
    if (cudaGetLastError() != cudaSuccess) return sfail(s, OD_ECUDA, "adam launch failed");
    return OD_OK;
}

const char* od_sur_last_error(const od_sur* s) { return s ? s->err.c_str() : g_sur_error.c_str(); }

int od_sur_set_gemm(od_sur* s, int engine)
{
    if (!s || (engine != OD_GEMM_TCGEN05 && engine != OD_GEMM_MMA_SYNC)) return sfail(s, OD_EINVAL, "bad engine");
    s->engine = engine;
    return OD_OK;
}

int od_gemm_bf16(const uint16_t* A, const uint16_t* B, const float* bias, float* C, uint16_t* Cb, int M, int N, int K,
                 int relu, int engine, int* err, void* stream)
{
    if (!A || !B || !C || !err || M < 1 || N < 16 || K < 16 || N % 16 || K % 16) return OD_EINVAL;
    if (engine != OD_GEMM_TCGEN05 && (engine != OD_GEMM_MMA_SYNC || M % 16)) return OD_EINVAL;
    const int e = gemm_bf16((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, bias, C, (__nv_bfloat16*)Cb, M, N, K,
                            relu, engine, err, (cudaStream_t)stream);
    return e == 0 ? OD_OK : OD_ECUDA;
}

}  // extern "C"
