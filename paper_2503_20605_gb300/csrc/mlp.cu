// mlp.cu -- the network of the learned warm start: a multilayer perceptron
// 3 -> 256 -> 256 -> 256 -> 64 (tanh hidden units, linear output) that maps
// (theta_eq, R0, lambda) to the equilibrium radial profile g(phi) = G(phi)/R0
// of the droplet about its centre (App. B parametrisation, 64 polar samples),
// trained by mean squared error with Adam.  The paper has no network; this
// is the warm start that shortens the runs to equilibrium.
//
// The 256-wide layers run on the fifth-generation tensor cores: BF16
// operands staged in shared memory in the canonical K-major core-matrix
// layout, tcgen05.mma issued by one thread, FP32 accumulators in tensor
// memory (TMEM), read back with tcgen05.ld for a fused epilogue (bias +
// tanh, bias, tanh' product, or plain store).  One CTA owns a 128-row tile
// of the output and the full width (N <= 256 columns of TMEM).  The input
// layer (K = 3) and the reductions run on the CUDA cores in FP32.
// Parameters: FP32 master copy + BF16 copies of the three tensor-core
// weight matrices, refreshed by the Adam kernel.
#include <math.h>
#include <string.h>

#include <cmath>

#include <string>
#include <vector>

#include "../../include/iblb.h"
#include "iblb_internal.h"

using namespace iblb;

namespace {

constexpr int NIN = 3, NH = 256, NOUT = 64;
constexpr int64_t NPARAM = (int64_t)NH * NIN + NH + 2 * ((int64_t)NH * NH + NH) + (int64_t)NOUT * NH + NOUT;
constexpr float BETA1 = 0.9f, BETA2 = 0.999f, ADAM_EPS = 1e-8f;

// ----------------------------------------------------------------- tcgen05
constexpr int TC_M = 128;        // output rows per CTA (M of one tcgen05.mma)
constexpr int TC_KC = 64;        // K elements staged per chunk (4 MMAs of K = 16)
constexpr int TC_THREADS = 128;  // 4 warps: warp w reads TMEM lanes 32w .. 32w + 31
constexpr int TC_A_BYTES = TC_M * TC_KC * 2;     // 16 KB
constexpr int TC_B_BYTES = 256 * TC_KC * 2;      // 32 KB (N <= 256)
// dynamic shared memory: A and B chunks plus the barrier and the TMEM slot,
// padded so that at most two CTAs share an SM (2 x 256 TMEM columns = all 512)
constexpr int TC_SMEM = 100 * 1024;
constexpr long long TC_WAIT_CYCLES = 1000000000LL;   // ~0.5 s: bounded barrier wait

enum Epi { EPI_TANH = 0, EPI_LINEAR = 1, EPI_DTANH = 2, EPI_STORE = 3 };

struct Gemm {
    // C (M x N) = A (M x K) . B (N x K)^T, FP32 accumulation
    int M, N, K;
    const __nv_bfloat16 *A;
    int64_t sam, sak;            // A(m, k) = A[m * sam + k * sak]
    const __nv_bfloat16 *B;
    int64_t sbn, sbk;            // B(n, k) = B[n * sbn + k * sbk]
    int epi;
    const float *bias;           // [N]           (EPI_TANH, EPI_LINEAR)
    const __nv_bfloat16 *h;      // [M x N], ld N (EPI_DTANH: multiply by 1 - h^2)
    float *of;                   // FP32 output, ld N (EPI_LINEAR, EPI_DTANH, EPI_STORE)
    __nv_bfloat16 *ob;           // BF16 output, ld N (EPI_TANH, EPI_DTANH)
    int *err;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05), no swizzle, K-major:
// start address, leading byte offset (between core matrices adjacent in K),
// stride byte offset (between 8-row groups in M or N), all in 16-byte
// units; descriptor version 1 at bits 46-47; swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D in F32, A and B in BF16, both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a staged operand chunk: 8 x 8 core
// matrices of 128 contiguous bytes (8 rows of 16 bytes), the 8 core matrices
// along K of one 8-row group contiguous (LBO = 128), row groups 1024 bytes
// apart (SBO = 1024)
__device__ __forceinline__ uint32_t core_off(int r, int kg) { return (r >> 3) * 1024 + kg * 128 + (r & 7) * 16; }

__device__ __forceinline__ void stage_operand(uint8_t *dst, const __nv_bfloat16 *src, int rows, int rows_pad,
                                              int64_t sr, int64_t sk, int k0, int K)
{
    // rows_pad x 8 vectors of 8 elements along K
    for (int v = threadIdx.x; v < rows_pad * (TC_KC / 8); v += TC_THREADS) {
        const int r = v >> 3, kg = v & 7;
        uint32_t w[4];
        for (int e = 0; e < 4; ++e) {
            const int ka = k0 + kg * 8 + 2 * e, kb = ka + 1;
            const unsigned short lo =
                (r < rows && ka < K) ? __bfloat16_as_ushort(src[(int64_t)r * sr + (int64_t)ka * sk]) : 0;
            const unsigned short hi =
                (r < rows && kb < K) ? __bfloat16_as_ushort(src[(int64_t)r * sr + (int64_t)kb * sk]) : 0;
            w[e] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint4 *>(dst + core_off(r, kg)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (clock64() - t0 > TC_WAIT_CYCLES)
            return false;
    }
}

__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(Gemm g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sa = smem;
    uint8_t *sb = smem + TC_A_BYTES;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + TC_A_BYTES + TC_B_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_M;
    const int rows_a = min(TC_M, g.M - m0);
    const int n_pad = (g.N + 15) & ~15;
    int ncols = 32;
    while (ncols < n_pad)
        ncols <<= 1;

    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(TC_M, n_pad);

    uint32_t phase = 0;
    for (int k0 = 0; k0 < g.K; k0 += TC_KC) {
        stage_operand(sa, g.A + (int64_t)m0 * g.sam, rows_a, TC_M, g.sam, g.sak, k0, g.K);
        stage_operand(sb, g.B, g.N, n_pad, g.sbn, g.sbk, k0, g.K);
        // generic-proxy writes of the operands become visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int ksteps = min(TC_KC, g.K - k0 + 15) / 16;
            for (int s = 0; s < ksteps && s < TC_KC / 16; ++s) {
                const uint64_t ad = smem_desc(smem_addr(sa) + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(smem_addr(sb) + s * 256, 128, 1024);
                const uint32_t acc = (k0 > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(bar))
                         : "memory");
        }
        // every thread waits for the MMAs of this chunk (the operands are
        // overwritten by the next chunk and TMEM is read after the last)
        const bool ok = mbar_wait_bounded(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                failed = 1;
                atomicExch(g.err, 1);
            }
            break;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (failed)   // give MMAs still in flight a bounded chance to finish before TMEM is freed
        mbar_wait_bounded(bar, phase ^ 1u);

    if (!failed) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < n_pad; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.M) {
                for (int e = 0; e < 16; ++e) {
                    const int col = c0 + e;
                    if (col >= g.N)
                        break;
                    const float acc = __uint_as_float(v[e]);
                    const int64_t o = (int64_t)row * g.N + col;
                    switch (g.epi) {
                    case EPI_TANH: g.ob[o] = __float2bfloat16_rn(tanhf(acc + g.bias[col])); break;
                    case EPI_LINEAR: g.of[o] = acc + g.bias[col]; break;
                    case EPI_DTANH: {
                        const float h = __bfloat162float(g.h[o]);
                        const float dz = acc * (1.0f - h * h);
                        g.of[o] = dz;
                        g.ob[o] = __float2bfloat16_rn(dz);
                        break;
                    }
                    default: g.of[o] = acc; break;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// --------------------------------------------------------- CUDA-core parts
// features of the raw inputs (theta_eq deg, R0, lambda), then the input layer
// h1 = tanh(W0 u + b0); one thread per (sample, unit)
__global__ void input_layer_kernel(const float *xraw, const int *idx, int S, const float *W0, const float *b0,
                                   float *u, __nv_bfloat16 *h1)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * NH)
        return;
    const int s = i / NH, o = i - s * NH;
    const int src = idx ? idx[s] : s;
    const float f0 = (xraw[3 * src] - 90.0f) / 70.0f;
    const float f1 = (xraw[3 * src + 1] - 16.0f) / 8.0f;
    const float f2 = log10f(xraw[3 * src + 2]);
    if (o == 0) {
        u[3 * s] = f0;
        u[3 * s + 1] = f1;
        u[3 * s + 2] = f2;
    }
    const float z = b0[o] + W0[3 * o] * f0 + W0[3 * o + 1] * f1 + W0[3 * o + 2] * f2;
    h1[i] = __float2bfloat16_rn(tanhf(z));
}

// d loss / d output = 2 (yhat - y) / (S * 64), in FP32 and BF16; per-sample
// squared errors for the loss
__global__ void loss_grad_kernel(const float *yhat, const float *y, const int *idx, int S, float *dy,
                                 __nv_bfloat16 *dyb, float *sq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * NOUT)
        return;
    const int s = i / NOUT, o = i - s * NOUT;
    const int src = idx ? idx[s] : s;
    const float d = yhat[i] - y[(int64_t)src * NOUT + o];
    const float g = 2.0f * d / (float)(S * NOUT);
    dy[i] = g;
    dyb[i] = __float2bfloat16_rn(g);
    sq[i] = d * d;
}

// Column sums over the batch in sample order (bias gradients), the input
// layer's weight gradient dW0 = d1^T u, and the loss (mean of sq); one warp
// per output, lanes stride over samples, fixed shuffle tree.
__global__ void reduce_grads_kernel(int S, const float *dy, const float *d3, const float *d2, const float *d1,
                                    const float *u, const float *sq, float *grad, double *loss)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    // outputs: gb3 (64), gb2 (256), gb1 (256), gb0 (256), gW0 (768), loss (1)
    const int nb3 = NOUT, nb = NH, nw0 = NH * NIN;
    const int total = nb3 + 3 * nb + nw0 + 1;
    if (w >= total)
        return;
    const int64_t off_W0 = 0, off_b0 = (int64_t)NH * NIN;
    const int64_t off_b1 = off_b0 + NH + (int64_t)NH * NH;
    const int64_t off_b2 = off_b1 + NH + (int64_t)NH * NH;
    const int64_t off_b3 = off_b2 + NH + (int64_t)NOUT * NH;
    float acc = 0.0f;
    double dacc = 0.0;
    int64_t dst;
    if (w < nb3) {
        for (int s = lane; s < S; s += 32) acc += dy[(int64_t)s * NOUT + w];
        dst = off_b3 + w;
    } else if (w < nb3 + nb) {
        const int o = w - nb3;
        for (int s = lane; s < S; s += 32) acc += d3[(int64_t)s * NH + o];
        dst = off_b2 + o;
    } else if (w < nb3 + 2 * nb) {
        const int o = w - nb3 - nb;
        for (int s = lane; s < S; s += 32) acc += d2[(int64_t)s * NH + o];
        dst = off_b1 + o;
    } else if (w < nb3 + 3 * nb) {
        const int o = w - nb3 - 2 * nb;
        for (int s = lane; s < S; s += 32) acc += d1[(int64_t)s * NH + o];
        dst = off_b0 + o;
    } else if (w < nb3 + 3 * nb + nw0) {
        const int q = w - nb3 - 3 * nb, o = q / NIN, i = q - o * NIN;
        for (int s = lane; s < S; s += 32) acc += d1[(int64_t)s * NH + o] * u[3 * s + i];
        dst = off_W0 + q;
    } else {
        for (int64_t k = lane; k < (int64_t)S * NOUT; k += 32) dacc += (double)sq[k];
        dst = -1;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    }
    if (lane == 0) {
        if (dst >= 0)
            grad[dst] = acc;
        else
            *loss = dacc / ((double)S * NOUT);
    }
}

// Adam step on the FP32 master parameters; refreshes the BF16 copies of the
// three tensor-core weight matrices
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, float lr, float c1, float c2,
                            __nv_bfloat16 *W1b, __nv_bfloat16 *W2b, __nv_bfloat16 *W3b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM)
        return;
    const float gi = g[i];
    const float mi = BETA1 * m[i] + (1.0f - BETA1) * gi;
    const float vi = BETA2 * v[i] + (1.0f - BETA2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + ADAM_EPS);
    p[i] = pi;
    const int64_t o1 = (int64_t)NH * NIN + NH, o2 = o1 + (int64_t)NH * NH + NH, o3 = o2 + (int64_t)NH * NH + NH;
    if (i >= o1 && i < o1 + (int64_t)NH * NH)
        W1b[i - o1] = __float2bfloat16_rn(pi);
    else if (i >= o2 && i < o2 + (int64_t)NH * NH)
        W2b[i - o2] = __float2bfloat16_rn(pi);
    else if (i >= o3 && i < o3 + (int64_t)NOUT * NH)
        W3b[i - o3] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        dst[i] = __float2bfloat16_rn(src[i]);
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct iblb_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0;
    int64_t t = 0;                       // Adam steps taken
    // parameters
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr;
    // activations (max_batch rows)
    float *x = nullptr, *y = nullptr, *u = nullptr, *yhat = nullptr, *dy = nullptr, *sq = nullptr;
    float *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;
    __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dyb = nullptr, *d3b = nullptr, *d2b = nullptr,
                  *d1b = nullptr;
    int *err = nullptr, *idx = nullptr;
    double *loss = nullptr;              // loss of each batch of an epoch (loss_cap entries)
    int loss_cap = 0;
    int64_t data_cap = 0;                // rows of x / y held on the device
    std::string msg;
};

namespace {

thread_local std::string g_mlp_error;

int mfail(iblb_mlp *m, int code, const std::string &s)
{
    if (m)
        m->msg = s;
    else
        g_mlp_error = s;
    return code;
}

#define MCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return mfail(m, IBLB_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

// parameter offsets
constexpr int64_t OFF_W0 = 0, OFF_B0 = (int64_t)NH * NIN;
constexpr int64_t OFF_W1 = OFF_B0 + NH, OFF_B1 = OFF_W1 + (int64_t)NH * NH;
constexpr int64_t OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + (int64_t)NH * NH;
constexpr int64_t OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + (int64_t)NOUT * NH;

cudaError_t gemm(iblb_mlp *mm, int M, int N, int K, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                 const __nv_bfloat16 *B, int64_t sbn, int64_t sbk, int epi, const float *bias,
                 const __nv_bfloat16 *h, float *of, __nv_bfloat16 *ob)
{
    Gemm g{M, N, K, A, sam, sak, B, sbn, sbk, epi, bias, h, of, ob, mm->err};
    tc_gemm_kernel<<<nblk(M, TC_M), TC_THREADS, TC_SMEM, mm->stream>>>(g);
    return cudaGetLastError();
}

// forward pass of S rows of x (device, raw inputs; rows idx[s] if idx)
cudaError_t forward(iblb_mlp *mm, const float *x, const int *idx, int S)
{
    input_layer_kernel<<<nblk((int64_t)S * NH, 256), 256, 0, mm->stream>>>(x, idx, S, mm->p + OFF_W0,
                                                                          mm->p + OFF_B0, mm->u, mm->h1);
    cudaError_t e;
    if ((e = gemm(mm, S, NH, NH, mm->h1, NH, 1, mm->W1b, NH, 1, EPI_TANH, mm->p + OFF_B1, nullptr, nullptr, mm->h2)))
        return e;
    if ((e = gemm(mm, S, NH, NH, mm->h2, NH, 1, mm->W2b, NH, 1, EPI_TANH, mm->p + OFF_B2, nullptr, nullptr, mm->h3)))
        return e;
    return gemm(mm, S, NOUT, NH, mm->h3, NH, 1, mm->W3b, NH, 1, EPI_LINEAR, mm->p + OFF_B3, nullptr, mm->yhat,
                nullptr);
}

// forward + backward: gradient of the mean squared error into mm->g, loss
// into mm->loss
cudaError_t forward_backward(iblb_mlp *mm, const float *x, const float *y, const int *idx, int S, double *loss)
{
    cudaError_t e;
    if ((e = forward(mm, x, idx, S)))
        return e;
    loss_grad_kernel<<<nblk((int64_t)S * NOUT, 256), 256, 0, mm->stream>>>(mm->yhat, y, idx, S, mm->dy, mm->dyb,
                                                                           mm->sq);
    float *g = mm->g;
    // layer 3: gW3 = dy^T h3 (64 x 256, K = S); d3 = (dy W3) * (1 - h3^2)
    if ((e = gemm(mm, NOUT, NH, S, mm->dyb, 1, NOUT, mm->h3, 1, NH, EPI_STORE, nullptr, nullptr, g + OFF_W3, nullptr)))
        return e;
    if ((e = gemm(mm, S, NH, NOUT, mm->dyb, NOUT, 1, mm->W3b, 1, NH, EPI_DTANH, nullptr, mm->h3, mm->d3, mm->d3b)))
        return e;
    // layer 2
    if ((e = gemm(mm, NH, NH, S, mm->d3b, 1, NH, mm->h2, 1, NH, EPI_STORE, nullptr, nullptr, g + OFF_W2, nullptr)))
        return e;
    if ((e = gemm(mm, S, NH, NH, mm->d3b, NH, 1, mm->W2b, 1, NH, EPI_DTANH, nullptr, mm->h2, mm->d2, mm->d2b)))
        return e;
    // layer 1
    if ((e = gemm(mm, NH, NH, S, mm->d2b, 1, NH, mm->h1, 1, NH, EPI_STORE, nullptr, nullptr, g + OFF_W1, nullptr)))
        return e;
    if ((e = gemm(mm, S, NH, NH, mm->d2b, NH, 1, mm->W1b, 1, NH, EPI_DTANH, nullptr, mm->h1, mm->d1, mm->d1b)))
        return e;
    const int nwarps = NOUT + 3 * NH + NH * NIN + 1;
    reduce_grads_kernel<<<nblk((int64_t)nwarps * 32, 256), 256, 0, mm->stream>>>(S, mm->dy, mm->d3, mm->d2, mm->d1,
                                                                                 mm->u, mm->sq, g, loss);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(iblb_mlp *mm)
{
    to_bf16_kernel<<<nblk((int64_t)NH * NH, 256), 256, 0, mm->stream>>>(mm->p + OFF_W1, mm->W1b, (int64_t)NH * NH);
    to_bf16_kernel<<<nblk((int64_t)NH * NH, 256), 256, 0, mm->stream>>>(mm->p + OFF_W2, mm->W2b, (int64_t)NH * NH);
    to_bf16_kernel<<<nblk((int64_t)NOUT * NH, 256), 256, 0, mm->stream>>>(mm->p + OFF_W3, mm->W3b,
                                                                          (int64_t)NOUT * NH);
    return cudaGetLastError();
}

int check_err(iblb_mlp *m)
{
    int h = 0;
    MCK(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    if (h) {
        MCK(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
        return mfail(m, IBLB_E_TIMEOUT, "a bounded wait for the tensor-core MMAs gave up");
    }
    return IBLB_OK;
}

int ensure_data(iblb_mlp *m, int64_t S)
{
    if (S <= m->data_cap)
        return IBLB_OK;
    if (m->x)
        MCK(cudaFree(m->x));
    if (m->y)
        MCK(cudaFree(m->y));
    m->x = m->y = nullptr;
    MCK(cudaMalloc((void **)&m->x, sizeof(float) * 3 * S));
    MCK(cudaMalloc((void **)&m->y, sizeof(float) * NOUT * S));
    m->data_cap = S;
    return IBLB_OK;
}

int upload(iblb_mlp *m, const double *x, const double *y, int64_t S)
{
    int r = ensure_data(m, S);
    if (r)
        return r;
    std::vector<float> hx(3 * S), hy(y ? NOUT * S : 0);
    for (int64_t i = 0; i < 3 * S; ++i)
        hx[i] = (float)x[i];
    for (int64_t i = 0; i < (int64_t)hy.size(); ++i)
        hy[i] = (float)y[i];
    MCK(cudaMemcpyAsync(m->x, hx.data(), sizeof(float) * hx.size(), cudaMemcpyHostToDevice, m->stream));
    if (y)
        MCK(cudaMemcpyAsync(m->y, hy.data(), sizeof(float) * hy.size(), cudaMemcpyHostToDevice, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return IBLB_OK;
}

bool inputs_valid(const double *x, int64_t S)
{
    for (int64_t s = 0; s < S; ++s)
        if (!(x[3 * s + 2] > 0.0) || !std::isfinite(x[3 * s]) || !std::isfinite(x[3 * s + 1]))
            return false;
    return true;
}

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int64_t iblb_mlp_param_count(void) { return NPARAM; }

const char *iblb_mlp_last_error(const iblb_mlp *m) { return m ? m->msg.c_str() : g_mlp_error.c_str(); }

int iblb_mlp_create(const float *params, int64_t n_params, int max_batch, void *stream, iblb_mlp **out)
{
    iblb_mlp *m = nullptr;
    if (!params || !out || n_params != NPARAM || max_batch < 1 || max_batch > (1 << 20))
        return mfail(nullptr, IBLB_E_ARG,
                     "iblb_mlp_create: need " + std::to_string(NPARAM) + " parameters and 1 <= max_batch <= 2^20");
    for (int64_t i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i]))
            return mfail(nullptr, IBLB_E_ARG, "iblb_mlp_create: non-finite parameter");
    m = new iblb_mlp();
    m->stream = (cudaStream_t)stream;
    m->max_batch = max_batch;
    const int64_t B = max_batch;
    auto fl = [&](float **p, int64_t n) { return cudaMalloc((void **)p, sizeof(float) * n); };
    auto bf = [&](__nv_bfloat16 **p, int64_t n) { return cudaMalloc((void **)p, sizeof(__nv_bfloat16) * n); };
    cudaError_t e = cudaSuccess;
    if (!e) e = fl(&m->p, NPARAM);
    if (!e) e = fl(&m->g, NPARAM);
    if (!e) e = fl(&m->m, NPARAM);
    if (!e) e = fl(&m->v, NPARAM);
    if (!e) e = bf(&m->W1b, (int64_t)NH * NH);
    if (!e) e = bf(&m->W2b, (int64_t)NH * NH);
    if (!e) e = bf(&m->W3b, (int64_t)NOUT * NH);
    if (!e) e = fl(&m->u, 3 * B);
    if (!e) e = fl(&m->yhat, NOUT * B);
    if (!e) e = fl(&m->dy, NOUT * B);
    if (!e) e = fl(&m->sq, NOUT * B);
    if (!e) e = fl(&m->d3, NH * B);
    if (!e) e = fl(&m->d2, NH * B);
    if (!e) e = fl(&m->d1, NH * B);
    if (!e) e = bf(&m->h1, NH * B);
    if (!e) e = bf(&m->h2, NH * B);
    if (!e) e = bf(&m->h3, NH * B);
    if (!e) e = bf(&m->dyb, NOUT * B);
    if (!e) e = bf(&m->d3b, NH * B);
    if (!e) e = bf(&m->d2b, NH * B);
    if (!e) e = bf(&m->d1b, NH * B);
    if (!e) e = cudaMalloc((void **)&m->err, sizeof(int));
    if (!e) e = cudaMalloc((void **)&m->idx, sizeof(int) * B);
    if (!e) e = cudaMalloc((void **)&m->loss, sizeof(double));
    if (!e) m->loss_cap = 1;
    if (!e) e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (!e) e = cudaMemcpyAsync(m->p, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream);
    if (!e) e = cudaMemsetAsync(m->m, 0, sizeof(float) * NPARAM, m->stream);
    if (!e) e = cudaMemsetAsync(m->v, 0, sizeof(float) * NPARAM, m->stream);
    if (!e) e = cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
    if (!e) e = refresh_bf16(m);
    if (!e) e = cudaStreamSynchronize(m->stream);
    if (e) {
        std::string s = std::string("iblb_mlp_create: ") + cudaGetErrorString(e);
        iblb_mlp_destroy(m);
        return mfail(nullptr, e == cudaErrorMemoryAllocation ? IBLB_E_NOMEM : IBLB_E_CUDA, s);
    }
    *out = m;
    return IBLB_OK;
}

void iblb_mlp_destroy(iblb_mlp *m)
{
    if (!m)
        return;
    void *ptrs[] = {m->p, m->g, m->m, m->v, m->W1b, m->W2b, m->W3b, m->x, m->y, m->u, m->yhat, m->dy, m->sq,
                    m->d3, m->d2, m->d1, m->h1, m->h2, m->h3, m->dyb, m->d3b, m->d2b, m->d1b, m->err, m->idx,
                    m->loss};
    for (void *p : ptrs)
        if (p)
            cudaFree(p);
    delete m;
}

int iblb_mlp_get_params(iblb_mlp *m, float *out, int64_t n)
{
    if (!m || !out || n != NPARAM)
        return mfail(m, IBLB_E_ARG, "iblb_mlp_get_params: bad arguments");
    MCK(cudaMemcpyAsync(out, m->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    return IBLB_OK;
}

int iblb_mlp_predict(iblb_mlp *m, const double *x, int S, double *y)
{
    if (!m || !x || !y || S < 1)
        return mfail(m, IBLB_E_ARG, "iblb_mlp_predict: bad arguments");
    if (!inputs_valid(x, S))
        return mfail(m, IBLB_E_ARG, "iblb_mlp_predict: inputs need finite theta_eq, R0 and lambda > 0");
    int r = upload(m, x, nullptr, S);
    if (r)
        return r;
    std::vector<float> hy((size_t)NOUT * m->max_batch);
    for (int s0 = 0; s0 < S; s0 += m->max_batch) {
        const int n = std::min(m->max_batch, S - s0);
        MCK(forward(m, m->x + 3 * (int64_t)s0, nullptr, n));
        MCK(cudaMemcpyAsync(hy.data(), m->yhat, sizeof(float) * NOUT * n, cudaMemcpyDeviceToHost, m->stream));
        MCK(cudaStreamSynchronize(m->stream));
        if ((r = check_err(m)))
            return r;
        for (int64_t i = 0; i < (int64_t)NOUT * n; ++i)
            y[(int64_t)NOUT * s0 + i] = hy[i];
    }
    return IBLB_OK;
}

int iblb_mlp_grad(iblb_mlp *m, const double *x, const double *y, int S, double *grad, double *loss)
{
    if (!m || !x || !y || !grad || !loss || S < 1 || S > m->max_batch)
        return mfail(m, IBLB_E_ARG, "iblb_mlp_grad: bad arguments (1 <= S <= max_batch)");
    if (!inputs_valid(x, S))
        return mfail(m, IBLB_E_ARG, "iblb_mlp_grad: inputs need finite theta_eq, R0 and lambda > 0");
    int r = upload(m, x, y, S);
    if (r)
        return r;
    MCK(forward_backward(m, m->x, m->y, nullptr, S, m->loss));
    std::vector<float> hg(NPARAM);
    MCK(cudaMemcpyAsync(hg.data(), m->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    MCK(cudaStreamSynchronize(m->stream));
    if ((r = check_err(m)))
        return r;
    for (int64_t i = 0; i < NPARAM; ++i)
        grad[i] = hg[i];
    return IBLB_OK;
}

int iblb_mlp_train(iblb_mlp *m, const double *x, const double *y, int S, int epochs, int batch, double lr,
                   uint64_t seed, double *loss_per_epoch)
{
    if (!m || !x || !y || S < 1 || epochs < 0 || batch < 1 || batch > m->max_batch || !(lr > 0.0))
        return mfail(m, IBLB_E_ARG, "iblb_mlp_train: bad arguments (1 <= batch <= max_batch, lr > 0)");
    if (!inputs_valid(x, S))
        return mfail(m, IBLB_E_ARG, "iblb_mlp_train: inputs need finite theta_eq, R0 and lambda > 0");
    int r = upload(m, x, y, S);
    if (r)
        return r;
    std::vector<int> perm(S);
    for (int i = 0; i < S; ++i)
        perm[i] = i;
    uint64_t st = seed;
    const int nb = S / batch;                  // full batches only
    if (nb > m->loss_cap) {
        MCK(cudaFree(m->loss));
        m->loss = nullptr;
        m->loss_cap = 0;
        MCK(cudaMalloc((void **)&m->loss, sizeof(double) * nb));
        m->loss_cap = nb;
    }
    std::vector<double> losses((size_t)std::max(nb, 1));
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = S - 1; i > 0; --i) {      // Fisher-Yates shuffle of the sample order
            const int j = (int)(splitmix(st) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        double ep_loss = 0.0;
        for (int b = 0; b < nb; ++b) {
            MCK(cudaMemcpyAsync(m->idx, perm.data() + (int64_t)b * batch, sizeof(int) * batch,
                                cudaMemcpyHostToDevice, m->stream));
            MCK(forward_backward(m, m->x, m->y, m->idx, batch, m->loss + b));
            m->t++;
            const float c1 = 1.0f - powf(BETA1, (float)m->t), c2 = 1.0f - powf(BETA2, (float)m->t);
            adam_kernel<<<nblk(NPARAM, 256), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, (float)lr, c1, c2, m->W1b,
                                                                  m->W2b, m->W3b);
            MCK(cudaGetLastError());
        }
        if (nb)
            MCK(cudaMemcpyAsync(losses.data(), m->loss, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
        MCK(cudaStreamSynchronize(m->stream));
        if ((r = check_err(m)))
            return r;
        for (int b = 0; b < nb; ++b)
            ep_loss += losses[b];
        if (loss_per_epoch)
            loss_per_epoch[ep] = nb ? ep_loss / nb : 0.0;
    }
    return IBLB_OK;
}

}  // extern "C"
