// Small multilayer perceptron for the learned warm start of a discharge:
// (U, p, L, C) -> cycle-averaged log-density profiles.  Weights bf16 (an
// fp32 master copy is what Adam updates), every product accumulated in fp32,
// tanh on the hidden layers, linear output; mean-squared-error loss.
//
// Shapes are tiny (widths of a few hundred, batches of a few hundred to a
// few thousand rows), so a training step is a chain of short launches: the
// contractions use a plain shared-memory-tiled FMA kernel with a fixed
// summation order (deterministic results), not the tensor cores, whose set-up
// would not pay at these sizes.
//
// Parameter layout (fp32 master, gradients, Adam moments): for each layer l,
// W_l as [in_l][out_l] row-major, then b_l[out_l].  The bf16 copy of the
// weights uses the same offsets.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <new>
#include <vector>

#include "internal.h"

namespace o2 {
namespace {

constexpr int GT = 64;          // output tile GT x GT per block
constexpr int GK = 16;          // k-slice staged in shared memory
constexpr int GTHREADS = 256;   // 16 x 16 threads, 4 x 4 outputs each

enum Epi { EPI_NONE = 0, EPI_TANH = 1, EPI_DTANH = 2 };

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[m][n] = epi( sum_k A(m,k) B(k,n) + bias[n] ), summed over k in order.
// A(m,k) = TA ? A[k lda + m] : A[m lda + k];  B(k,n) = TB ? B[n ldb + k] : B[k ldb + n].
// EPI_TANH: tanh of the sum; EPI_DTANH: the sum times (1 - H[m][n]^2).
template <bool TA, bool TB, typename BT>
__global__ void __launch_bounds__(GTHREADS) k_gemm(const float* __restrict__ A, int lda, const BT* __restrict__ B,
                                                   int ldb, float* __restrict__ C, int ldc, int M, int N, int K,
                                                   const float* __restrict__ bias, int epi,
                                                   const float* __restrict__ H) {
    __shared__ float As[GK][GT + 1];
    __shared__ float Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += GTHREADS) {
            int mm, kk;
            if (TA) { kk = e / GT; mm = e % GT; } else { mm = e / GK; kk = e % GK; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.0f;
        }
        for (int e = threadIdx.x; e < GT * GK; e += GTHREADS) {
            int nn, kk;
            if (TB) { nn = e / GK; kk = e % GK; } else { kk = e / GT; nn = e % GT; }
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < K) ? (TB ? ldf(&B[(size_t)n * ldb + k]) : ldf(&B[(size_t)k * ldb + n])) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (bias) v += bias[n];
            if (epi == EPI_TANH) v = tanhf(v);
            else if (epi == EPI_DTANH) { const float h = H[(size_t)m * N + n]; v = v * (1.0f - h * h); }
            C[(size_t)m * ldc + n] = v;
        }
    }
}

// dY = 2 (Y - T) / (B N); per-block partial sums of (Y - T)^2 (fixed order).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY, size_t n,
                      float scale, float* __restrict__ partial) {
    __shared__ float red[256];
    float s = 0.0f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.0f * d * scale;
        s = fmaf(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const float* __restrict__ partial, int nb, float scale, float* loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < nb; ++i) s += partial[i];
        *loss = s * scale;
    }
}

// db[n] = sum_m dZ[m][n] (one thread per column, rows in order).
__global__ void k_colsum(const float* __restrict__ dZ, int M, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += dZ[(size_t)m * N + n];
    db[n] = s;
}

// Adam (Kingma & Ba 2015) on the fp32 master parameters, then the bf16 copy
// of the weights (entries flagged in is_w).
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ Mo,
                       float* __restrict__ Ve, __nv_bfloat16* __restrict__ Wb, const unsigned char* __restrict__ is_w,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = fmaf(b1, Mo[i], (1.0f - b1) * g);
        const float v = fmaf(b2, Ve[i], (1.0f - b2) * g * g);
        Mo[i] = m;
        Ve[i] = v;
        const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        P[i] = p;
        if (is_w[i]) Wb[i] = __float2bfloat16_rn(p);
    }
}

__global__ void k_to_bf16(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wb,
                          const unsigned char* __restrict__ is_w, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (is_w[i]) Wb[i] = __float2bfloat16_rn(P[i]);
}

template <bool TA, bool TB, typename BT>
void gemm(const float* A, int lda, const BT* B, int ldb, float* C, int ldc, int M, int N, int K, const float* bias,
          int epi, const float* H, cudaStream_t s) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm<TA, TB, BT><<<grid, GTHREADS, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, bias, epi, H);
}

}  // namespace
}  // namespace o2

using namespace o2;

struct o2pic_mlp {
    int device = 0;
    std::vector<int> w;                    // widths, w[0] = inputs, w[L] = outputs
    std::vector<size_t> offW, offB;        // parameter offsets per layer
    size_t nparams = 0;
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Ve = nullptr;
    __nv_bfloat16* Wb = nullptr;
    unsigned char* is_w = nullptr;
    // activations for a batch of up to cap rows: H[l] (l = 1..L-1), Y, dZ ping-pong
    int cap = 0;
    std::vector<float*> H;
    float *Y = nullptr, *dA = nullptr, *dB = nullptr, *partial = nullptr;
    unsigned long long t = 0;              // Adam steps taken
};

namespace {

constexpr int MSE_BLOCKS = 120;

int layers(const o2pic_mlp* m) { return (int)m->w.size() - 1; }

void free_acts(o2pic_mlp* m) {
    for (float* h : m->H) if (h) cudaFree(h);
    m->H.clear();
    if (m->Y) cudaFree(m->Y);
    if (m->dA) cudaFree(m->dA);
    if (m->dB) cudaFree(m->dB);
    m->Y = m->dA = m->dB = nullptr;
    m->cap = 0;
}

int ensure_acts(o2pic_mlp* m, int B) {
    if (B <= m->cap) return O2PIC_OK;
    free_acts(m);
    int wmax = 0;
    for (int x : m->w) wmax = std::max(wmax, x);
    const int L = layers(m);
    m->H.assign(L, nullptr);
    for (int l = 1; l < L; ++l)
        if (cudaMalloc((void**)&m->H[l], sizeof(float) * (size_t)B * m->w[l]) != cudaSuccess) return O2PIC_E_CUDA;
    if (cudaMalloc((void**)&m->Y, sizeof(float) * (size_t)B * m->w[L]) != cudaSuccess) return O2PIC_E_CUDA;
    if (cudaMalloc((void**)&m->dA, sizeof(float) * (size_t)B * wmax) != cudaSuccess) return O2PIC_E_CUDA;
    if (cudaMalloc((void**)&m->dB, sizeof(float) * (size_t)B * wmax) != cudaSuccess) return O2PIC_E_CUDA;
    m->cap = B;
    return O2PIC_OK;
}

// Forward pass of B rows of X into m->H and out (the output layer).
void forward(o2pic_mlp* m, const float* X, float* out, int B, cudaStream_t s) {
    const int L = layers(m);
    const float* in = X;
    for (int l = 1; l <= L; ++l) {
        const int K = m->w[l - 1], N = m->w[l];
        float* dst = (l == L) ? out : m->H[l];
        gemm<false, false>(in, K, m->Wb + m->offW[l - 1], N, dst, N, B, N, K, m->P + m->offB[l - 1],
                           l == L ? EPI_NONE : EPI_TANH, nullptr, s);
        in = dst;
    }
}

// Loss and gradients of the mean-squared error over B rows into m->G.
void backward(o2pic_mlp* m, const float* X, const float* T, int B, float* loss, cudaStream_t s) {
    const int L = layers(m);
    const size_t nout = (size_t)B * m->w[L];
    const float scale = 1.0f / (float)nout;
    k_mse<<<MSE_BLOCKS, 256, 0, s>>>(m->Y, T, m->dA, nout, scale, m->partial);
    k_loss_final<<<1, 32, 0, s>>>(m->partial, MSE_BLOCKS, scale, loss);
    float* dZ = m->dA;     // gradient at the pre-activation of layer l
    float* dN = m->dB;
    for (int l = L; l >= 1; --l) {
        const int K = m->w[l - 1], N = m->w[l];
        const float* Hin = (l == 1) ? X : m->H[l - 1];
        // dW_l = H_{l-1}^T dZ_l   ([K][N]);  db_l = column sums of dZ_l
        gemm<true, false>(Hin, K, dZ, N, m->G + m->offW[l - 1], N, K, N, B, nullptr, EPI_NONE, nullptr, s);
        k_colsum<<<(N + 127) / 128, 128, 0, s>>>(dZ, B, N, m->G + m->offB[l - 1]);
        if (l > 1) {
            // dZ_{l-1} = (dZ_l W_l^T) (1 - H_{l-1}^2)
            gemm<false, true>(dZ, N, m->Wb + m->offW[l - 1], N, dN, K, B, K, N, nullptr, EPI_DTANH, m->H[l - 1], s);
            std::swap(dZ, dN);
        }
    }
}

// SplitMix64 (Steele, Lea & Flood 2014) for the initial weights.
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int o2pic_mlp_create(const int32_t* widths, int32_t n_widths, uint64_t seed, o2pic_mlp** out) {
    if (!out) return O2PIC_E_INVALID_ARG;
    *out = nullptr;
    if (!widths || n_widths < 2 || n_widths > 16) return O2PIC_E_INVALID_ARG;
    for (int i = 0; i < n_widths; ++i)
        if (widths[i] < 1 || widths[i] > 8192) return O2PIC_E_INVALID_ARG;
    o2pic_mlp* m = new (std::nothrow) o2pic_mlp;
    if (!m) return O2PIC_E_CUDA;
    cudaGetDevice(&m->device);
    m->w.assign(widths, widths + n_widths);
    const int L = n_widths - 1;
    for (int l = 0; l < L; ++l) {
        m->offW.push_back(m->nparams);
        m->nparams += (size_t)m->w[l] * m->w[l + 1];
        m->offB.push_back(m->nparams);
        m->nparams += (size_t)m->w[l + 1];
    }
    // Glorot-uniform weights U(-a, a), a = sqrt(6 / (in + out)); zero biases
    std::vector<float> P(m->nparams, 0.0f);
    std::vector<unsigned char> isw(m->nparams, 0);
    uint64_t st = seed;
    for (int l = 0; l < L; ++l) {
        const double a = std::sqrt(6.0 / (double)(m->w[l] + m->w[l + 1]));
        const size_t n = (size_t)m->w[l] * m->w[l + 1];
        for (size_t i = 0; i < n; ++i) {
            const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            P[m->offW[l] + i] = (float)((2.0 * u - 1.0) * a);
            isw[m->offW[l] + i] = 1;
        }
    }
    bool ok = cudaMalloc((void**)&m->P, sizeof(float) * m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->G, sizeof(float) * m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->Mo, sizeof(float) * m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->Ve, sizeof(float) * m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->Wb, sizeof(__nv_bfloat16) * m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->is_w, m->nparams) == cudaSuccess &&
              cudaMalloc((void**)&m->partial, sizeof(float) * MSE_BLOCKS) == cudaSuccess;
    ok = ok && cudaMemcpy(m->is_w, isw.data(), m->nparams, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(m->G, 0, sizeof(float) * m->nparams) == cudaSuccess &&
         cudaMemset(m->Mo, 0, sizeof(float) * m->nparams) == cudaSuccess &&
         cudaMemset(m->Ve, 0, sizeof(float) * m->nparams) == cudaSuccess &&
         cudaMemset(m->Wb, 0, sizeof(__nv_bfloat16) * m->nparams) == cudaSuccess;
    if (!ok) { o2pic_mlp_destroy(m); return O2PIC_E_CUDA; }
    *out = m;
    return o2pic_mlp_set_params(m, P.data());
}

uint64_t o2pic_mlp_num_params(o2pic_mlp* m) { return m ? m->nparams : 0; }

int o2pic_mlp_set_params(o2pic_mlp* m, const float* host) {
    if (!m || !host) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return O2PIC_E_CUDA;
    if (cudaMemcpy(m->P, host, sizeof(float) * m->nparams, cudaMemcpyHostToDevice) != cudaSuccess) return O2PIC_E_CUDA;
    k_to_bf16<<<120, 256>>>(m->P, m->Wb, m->is_w, m->nparams);
    if (cudaDeviceSynchronize() != cudaSuccess) return O2PIC_E_CUDA;
    m->t = 0;
    cudaMemset(m->Mo, 0, sizeof(float) * m->nparams);
    cudaMemset(m->Ve, 0, sizeof(float) * m->nparams);
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

int o2pic_mlp_get_params(o2pic_mlp* m, float* host) {
    if (!m || !host) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return O2PIC_E_CUDA;
    return cudaMemcpy(host, m->P, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost) == cudaSuccess ? O2PIC_OK
                                                                                                   : O2PIC_E_CUDA;
}

int o2pic_mlp_forward(o2pic_mlp* m, const float* X, float* Y, int32_t B, void* stream) {
    if (!m || B < 0 || (B > 0 && (!X || !Y))) return O2PIC_E_INVALID_ARG;
    if (B == 0) return O2PIC_OK;
    if (cudaSetDevice(m->device) != cudaSuccess) return O2PIC_E_CUDA;
    if (int rc = ensure_acts(m, B)) return rc;
    forward(m, X, Y, B, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

int o2pic_mlp_gradients(o2pic_mlp* m, const float* X, const float* T, int32_t B, float* grad, float* loss,
                        void* stream) {
    if (!m || B < 1 || !X || !T || !loss) return O2PIC_E_INVALID_ARG;
    if (cudaSetDevice(m->device) != cudaSuccess) return O2PIC_E_CUDA;
    if (int rc = ensure_acts(m, B)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    forward(m, X, m->Y, B, s);
    backward(m, X, T, B, loss, s);
    if (grad && cudaMemcpyAsync(grad, m->G, sizeof(float) * m->nparams, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return O2PIC_E_CUDA;
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

int o2pic_mlp_train_step(o2pic_mlp* m, const float* X, const float* T, int32_t B, float lr, float* loss,
                         void* stream) {
    if (!m || B < 1 || !X || !T || !loss || !(lr >= 0.0f)) return O2PIC_E_INVALID_ARG;
    if (int rc = o2pic_mlp_gradients(m, X, T, B, nullptr, loss, stream)) return rc;
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)m->t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)m->t));
    k_adam<<<120, 256, 0, (cudaStream_t)stream>>>(m->P, m->G, m->Mo, m->Ve, m->Wb, m->is_w, m->nparams, lr, b1, b2,
                                                  1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? O2PIC_OK : O2PIC_E_CUDA;
}

void o2pic_mlp_destroy(o2pic_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    free_acts(m);
    for (void* p : {(void*)m->P, (void*)m->G, (void*)m->Mo, (void*)m->Ve, (void*)m->Wb, (void*)m->is_w,
                    (void*)m->partial})
        if (p) cudaFree(p);
    delete m;
}

}  // extern "C"
