// Tile-planner network: an 8 -> 64 -> 64 -> 2 multilayer perceptron (ReLU, FP32) with
// hand-written forward, backward and Adam kernels, trained on the GPU from autotuner
// timings (planner.cpp uses it for OC_PLAN_LEARNED).
//
// Parameter vector layout (OC_MLP_NPARAMS floats): W1[64][8], b1[64], W2[64][64], b2[64],
// W3[2][64], b3[2]. Loss over n samples: L = 1/(2n) sum_i sum_k (y_ik - t_ik)^2.
// Every sum runs in a fixed order (one thread per output element, sequential over its
// inputs), so results do not depend on the launch configuration.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/oc.h"
#include "mlp.h"

namespace oc {

namespace {

constexpr int kIn = 8, kH = 64, kOut = 2;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kN = ob3 + kOut;
static_assert(kN == 4866, "parameter layout");

// Z[i][o] = b[o] + sum_j W[o][j] X[i][j];  A = relu(Z) or Z
__global__ void k_dense(const float* __restrict__ W, const float* __restrict__ b, const float* __restrict__ X,
                        int n, int in, int out, int relu, float* __restrict__ Z, float* __restrict__ A)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * out) return;
    const int i = t / out, o = t % out;
    float z = b[o];
    for (int j = 0; j < in; ++j) z = __fmaf_rn(W[o * in + j], X[i * in + j], z);
    Z[t] = z;
    A[t] = relu ? fmaxf(z, 0.0f) : z;
}

// dZ[i][k] = (Y[i][k] - T[i][k]) / n   (output layer, squared loss)
__global__ void k_out_grad(const float* Y, const float* T, int n, int out, float* dZ)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * out) return;
    dZ[t] = (Y[t] - T[t]) / (float)n;
}

// dW[o][j] = sum_i dZ[i][o] A[i][j]; db[o] = sum_i dZ[i][o]
__global__ void k_wgrad(const float* __restrict__ dZ, const float* __restrict__ A, int n, int out, int in,
                        float* __restrict__ dW, float* __restrict__ db)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= out * (in + 1)) return;
    const int o = t / (in + 1), j = t % (in + 1);
    float s = 0.0f;
    if (j < in)
        for (int i = 0; i < n; ++i) s = __fmaf_rn(dZ[i * out + o], A[i * in + j], s);
    else
        for (int i = 0; i < n; ++i) s += dZ[i * out + o];
    if (j < in) dW[o * in + j] = s;
    else db[o] = s;
}

// dZp[i][j] = (sum_k W[k][j] dZ[i][k]) * (Zp[i][j] > 0)   (back through a ReLU layer)
__global__ void k_backprop(const float* __restrict__ W, const float* __restrict__ dZ, const float* __restrict__ Zp,
                           int n, int out, int in, float* __restrict__ dZp)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * in) return;
    const int i = t / in, j = t % in;
    float s = 0.0f;
    for (int k = 0; k < out; ++k) s = __fmaf_rn(W[k * in + j], dZ[i * out + k], s);
    dZp[t] = Zp[t] > 0.0f ? s : 0.0f;
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    m[t] = b1 * m[t] + (1.0f - b1) * gt;
    v[t] = b2 * v[t] + (1.0f - b2) * gt * gt;
    const float mh = m[t] / c1, vh = v[t] / c2;
    p[t] = p[t] - lr * mh / (sqrtf(vh) + eps);
}

inline int blocks(int n) { return (n + 127) / 128; }

}  // namespace

// Device workspace for n samples (activations and gradients).
struct MlpWork {
    int n = 0;
    float *X = nullptr, *T = nullptr, *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *Z3 = nullptr,
          *Y = nullptr, *dZ3 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    cudaError_t alloc(int n_)
    {
        n = n_;
        size_t f = sizeof(float);
        float** bufs[] = {&X, &T, &Z1, &A1, &Z2, &A2, &Z3, &Y, &dZ3, &dZ2, &dZ1, &P, &G, &M, &V};
        size_t sz[] = {(size_t)n * kIn, (size_t)n * kOut, (size_t)n * kH, (size_t)n * kH, (size_t)n * kH,
                       (size_t)n * kH, (size_t)n * kOut, (size_t)n * kOut, (size_t)n * kOut, (size_t)n * kH,
                       (size_t)n * kH, (size_t)kN, (size_t)kN, (size_t)kN, (size_t)kN};
        for (int k = 0; k < 15; ++k) {
            cudaError_t e = cudaMalloc((void**)bufs[k], std::max<size_t>(1, sz[k]) * f);
            if (e != cudaSuccess) return e;
        }
        cudaMemset(M, 0, kN * f);
        cudaMemset(V, 0, kN * f);
        return cudaSuccess;
    }
    ~MlpWork()
    {
        float* bufs[] = {X, T, Z1, A1, Z2, A2, Z3, Y, dZ3, dZ2, dZ1, P, G, M, V};
        for (float* b : bufs)
            if (b) cudaFree(b);
    }
};

static void forward(MlpWork& w, cudaStream_t s)
{
    const int n = w.n;
    k_dense<<<blocks(n * kH), 128, 0, s>>>(w.P + oW1, w.P + ob1, w.X, n, kIn, kH, 1, w.Z1, w.A1);
    k_dense<<<blocks(n * kH), 128, 0, s>>>(w.P + oW2, w.P + ob2, w.A1, n, kH, kH, 1, w.Z2, w.A2);
    k_dense<<<blocks(n * kOut), 128, 0, s>>>(w.P + oW3, w.P + ob3, w.A2, n, kH, kOut, 0, w.Z3, w.Y);
}

static void backward(MlpWork& w, cudaStream_t s)
{
    const int n = w.n;
    k_out_grad<<<blocks(n * kOut), 128, 0, s>>>(w.Y, w.T, n, kOut, w.dZ3);
    k_wgrad<<<blocks(kOut * (kH + 1)), 128, 0, s>>>(w.dZ3, w.A2, n, kOut, kH, w.G + oW3, w.G + ob3);
    k_backprop<<<blocks(n * kH), 128, 0, s>>>(w.P + oW3, w.dZ3, w.Z2, n, kOut, kH, w.dZ2);
    k_wgrad<<<blocks(kH * (kH + 1)), 128, 0, s>>>(w.dZ2, w.A1, n, kH, kH, w.G + oW2, w.G + ob2);
    k_backprop<<<blocks(n * kH), 128, 0, s>>>(w.P + oW2, w.dZ2, w.Z1, n, kH, kH, w.dZ1);
    k_wgrad<<<blocks(kH * (kIn + 1)), 128, 0, s>>>(w.dZ1, w.X, n, kH, kIn, w.G + oW1, w.G + ob1);
}

static double host_loss(const std::vector<float>& Y, const float* T, int n)
{
    double l = 0;
    for (int i = 0; i < n * kOut; ++i) {
        const double d = (double)Y[i] - (double)T[i];
        l += d * d;
    }
    return l / (2.0 * n);
}

int mlp_nparams() { return kN; }

cudaError_t mlp_forward(const float* params, const float* X, int n, float* Y)
{
    MlpWork w;
    cudaError_t e = w.alloc(n);
    if (e != cudaSuccess) return e;
    cudaMemcpy(w.P, params, kN * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(w.X, X, (size_t)n * kIn * sizeof(float), cudaMemcpyHostToDevice);
    forward(w, 0);
    e = cudaMemcpy(Y, w.Y, (size_t)n * kOut * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t mlp_loss_grad(const float* params, const float* X, const float* T, int n, float* grad, double* loss)
{
    MlpWork w;
    cudaError_t e = w.alloc(n);
    if (e != cudaSuccess) return e;
    cudaMemcpy(w.P, params, kN * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(w.X, X, (size_t)n * kIn * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(w.T, T, (size_t)n * kOut * sizeof(float), cudaMemcpyHostToDevice);
    forward(w, 0);
    backward(w, 0);
    e = cudaMemcpy(grad, w.G, kN * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    std::vector<float> Y((size_t)n * kOut);
    e = cudaMemcpy(Y.data(), w.Y, Y.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (loss) *loss = host_loss(Y, T, n);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

cudaError_t mlp_train(float* params, const float* X, const float* T, int n, int epochs, float lr,
                      float* loss_hist)
{
    MlpWork w;
    cudaError_t e = w.alloc(n);
    if (e != cudaSuccess) return e;
    cudaMemcpy(w.P, params, kN * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(w.X, X, (size_t)n * kIn * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(w.T, T, (size_t)n * kOut * sizeof(float), cudaMemcpyHostToDevice);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double c1 = 1.0, c2 = 1.0;
    std::vector<float> Y((size_t)n * kOut);
    for (int ep = 0; ep < epochs; ++ep) {
        forward(w, 0);
        if (loss_hist) {
            cudaMemcpy(Y.data(), w.Y, Y.size() * sizeof(float), cudaMemcpyDeviceToHost);
            loss_hist[ep] = (float)host_loss(Y, T, n);
        }
        backward(w, 0);
        c1 *= b1;
        c2 *= b2;
        k_adam<<<blocks(kN), 128>>>(w.P, w.G, w.M, w.V, kN, lr, b1, b2, eps, (float)(1.0 - c1), (float)(1.0 - c2));
    }
    e = cudaMemcpy(params, w.P, kN * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace oc
