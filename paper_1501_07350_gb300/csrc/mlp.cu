// mlp.cu -- the learned cost model of the run-time tuner: a small multilayer
// perceptron, trained and evaluated on the GPU by the kernels in this file.
//
// The paper's auto-tuner (Sec. 3.2.3) times every communication method at
// initialisation and keeps the fastest; here the tuner's timings become a
// dataset, and a network y = f(features of (problem, candidate)) predicts the
// logarithm of a candidate's time, so a plan can pick a candidate without
// running all of them (openfft_set_tuning(..., OPENFFT_TUNE_LEARNED, ...)).
//
// Network: d inputs -> H tanh -> H tanh -> 1 linear.  Parameters, flat float
// array: W1[d][H], b1[H], W2[H][H], b2[H], W3[H], b3.  Loss: mean squared
// error over n samples.  Optimiser: Adam.  Training runs full-batch steps;
// one step (forward, loss gradient, backward, Adam) is captured once in a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/openfft_gb.h"

namespace ofg {
int set_last_error(int status, const char* msg);   // capi.cu
}

using namespace ofg;

namespace {

constexpr int kThreads = 256;

// Y[s][j] = act(sum_i X[s][i] W[i][j] + b[j]); act = tanh or identity
__global__ void dense_forward(const float* __restrict__ X, const float* __restrict__ W,
                              const float* __restrict__ b, float* __restrict__ Y, int n, int k, int m,
                              int use_tanh)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * m) return;
    const int s = idx / m, j = idx - s * m;
    float z = b[j];
    for (int i = 0; i < k; ++i) z = fmaf(X[s * k + i], W[i * m + j], z);
    Y[idx] = use_tanh ? tanhf(z) : z;
}

// dZ = dY * act'(Z) with tanh'(Z) = 1 - Y^2 (Y = tanh Z), in place on dY
__global__ void act_backward(float* __restrict__ dY, const float* __restrict__ Y, int total)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const float y = Y[idx];
    dY[idx] *= 1.f - y * y;
}

// dW[i][j] = sum_s X[s][i] dZ[s][j]; db[j] = sum_s dZ[s][j]  (one thread per (i, j) / j)
__global__ void dense_grad_w(const float* __restrict__ X, const float* __restrict__ dZ,
                             float* __restrict__ dW, float* __restrict__ db, int n, int k, int m)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < k * m) {
        const int i = idx / m, j = idx - i * m;
        float acc = 0.f;
        for (int s = 0; s < n; ++s) acc = fmaf(X[s * k + i], dZ[s * m + j], acc);
        dW[idx] = acc;
    } else if (idx < k * m + m) {
        const int j = idx - k * m;
        float acc = 0.f;
        for (int s = 0; s < n; ++s) acc += dZ[s * m + j];
        db[j] = acc;
    }
}

// dX[s][i] = sum_j dZ[s][j] W[i][j]
__global__ void dense_grad_x(const float* __restrict__ dZ, const float* __restrict__ W,
                             float* __restrict__ dX, int n, int k, int m)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int s = idx / k, i = idx - s * k;
    float acc = 0.f;
    for (int j = 0; j < m; ++j) acc = fmaf(dZ[s * m + j], W[i * m + j], acc);
    dX[idx] = acc;
}

// dY = 2 (yhat - y) / n; loss = mean (yhat - y)^2 (one block reduces)
__global__ void mse_grad(const float* __restrict__ yhat, const float* __restrict__ y, float* __restrict__ dY,
                         float* __restrict__ loss, int n)
{
    __shared__ float red[kThreads];
    float acc = 0.f;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const float d = yhat[s] - y[s];
        dY[s] = 2.f * d / (float)n;
        acc = fmaf(d, d, acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)n;
}

// Adam (Kingma & Ba): m = b1 m + (1 - b1) g; v = b2 v + (1 - b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps); t is read from
// device memory and advanced by the last thread so a captured step can replay.
__global__ void adam_step(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int* __restrict__ t, int np, float lr, float b1, float b2,
                          float eps)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int step = *t + 1;
    if (idx < np) {
        const float gi = g[idx];
        const float mi = b1 * m[idx] + (1.f - b1) * gi;
        const float vi = b2 * v[idx] + (1.f - b2) * gi * gi;
        m[idx] = mi;
        v[idx] = vi;
        const float mh = mi / (1.f - powf(b1, (float)step));
        const float vh = vi / (1.f - powf(b2, (float)step));
        p[idx] -= lr * mh / (sqrtf(vh) + eps);
    }
}

__global__ void advance_step(int* t) { *t += 1; }

unsigned blocks(int n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct Net {
    int d, H, n;
    // device buffers
    float *X = nullptr, *y = nullptr, *h1 = nullptr, *h2 = nullptr, *yh = nullptr;
    float *dy = nullptr, *dh2 = nullptr, *dh1 = nullptr;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    int* t = nullptr;
    int np() const { return d * H + H + H * H + H + H + 1; }
    // parameter views
    float* W1(float* q) const { return q; }
    float* b1(float* q) const { return q + d * H; }
    float* W2(float* q) const { return q + d * H + H; }
    float* b2(float* q) const { return q + d * H + H + H * H; }
    float* W3(float* q) const { return q + d * H + H + H * H + H; }
    float* b3(float* q) const { return q + d * H + H + H * H + H + H; }
};

void net_free(Net& N)
{
    float* bufs[] = {N.X, N.y, N.h1, N.h2, N.yh, N.dy, N.dh2, N.dh1, N.p, N.g, N.m, N.v, N.loss};
    for (float* b : bufs) cudaFree(b);
    cudaFree(N.t);
}

int net_alloc(Net& N, int d, int H, int n, bool train)
{
    N.d = d; N.H = H; N.n = n;
    const size_t np = (size_t)N.np();
    cudaError_t e = cudaSuccess;
    auto A = [&](float** q, size_t cnt) { if (!e) e = cudaMalloc(q, cnt * sizeof(float)); };
    A(&N.X, (size_t)n * d); A(&N.h1, (size_t)n * H); A(&N.h2, (size_t)n * H); A(&N.yh, (size_t)n);
    A(&N.p, np);
    if (train) {
        A(&N.y, (size_t)n); A(&N.dy, (size_t)n); A(&N.dh2, (size_t)n * H); A(&N.dh1, (size_t)n * H);
        A(&N.g, np); A(&N.m, np); A(&N.v, np); A(&N.loss, 1);
        if (!e) e = cudaMalloc(&N.t, sizeof(int));
    }
    if (e) { cudaGetLastError(); net_free(N); return set_last_error(OPENFFT_ERR_NOMEM, "cost-model buffers"); }
    return OPENFFT_OK;
}

void forward(const Net& N, cudaStream_t s)
{
    dense_forward<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.X, N.W1(N.p), N.b1(N.p), N.h1, N.n, N.d, N.H, 1);
    dense_forward<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.h1, N.W2(N.p), N.b2(N.p), N.h2, N.n, N.H, N.H, 1);
    dense_forward<<<blocks(N.n), kThreads, 0, s>>>(N.h2, N.W3(N.p), N.b3(N.p), N.yh, N.n, N.H, 1, 0);
}

void backward(const Net& N, cudaStream_t s)
{
    mse_grad<<<1, kThreads, 0, s>>>(N.yh, N.y, N.dy, N.loss, N.n);
    // layer 3 (linear): dW3, db3, dh2
    dense_grad_w<<<blocks(N.H + 1), kThreads, 0, s>>>(N.h2, N.dy, N.W3(N.g), N.b3(N.g), N.n, N.H, 1);
    dense_grad_x<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.dy, N.W3(N.p), N.dh2, N.n, N.H, 1);
    // layer 2 (tanh)
    act_backward<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.dh2, N.h2, N.n * N.H);
    dense_grad_w<<<blocks(N.H * N.H + N.H), kThreads, 0, s>>>(N.h1, N.dh2, N.W2(N.g), N.b2(N.g), N.n, N.H, N.H);
    dense_grad_x<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.dh2, N.W2(N.p), N.dh1, N.n, N.H, N.H);
    // layer 1 (tanh)
    act_backward<<<blocks(N.n * N.H), kThreads, 0, s>>>(N.dh1, N.h1, N.n * N.H);
    dense_grad_w<<<blocks(N.d * N.H + N.H), kThreads, 0, s>>>(N.X, N.dh1, N.W1(N.g), N.b1(N.g), N.n, N.d, N.H);
}

int check_dims(int d, int H, int n)
{
    if (d < 1 || d > 256 || H < 1 || H > 256 || n < 1 || n > (1 << 20))
        return set_last_error(OPENFFT_ERR_INVALID_ARG, "cost model needs 1 <= d, H <= 256 and 1 <= n <= 2^20");
    return OPENFFT_OK;
}

int cuda_status(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e) return set_last_error(OPENFFT_ERR_CUDA, what);
    return OPENFFT_OK;
}

}  // namespace

extern "C" {

int openfft_mlp_num_params(int d, int hidden) { return d * hidden + hidden + hidden * hidden + hidden + hidden + 1; }

int openfft_mlp_predict(int d, int hidden, const float* params, const float* X, int n, float* yhat)
{
    if (!params || !X || !yhat) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null pointer");
    int st = check_dims(d, hidden, n);
    if (st) return st;
    Net N;
    if ((st = net_alloc(N, d, hidden, n, false))) return st;
    cudaMemcpy(N.p, params, sizeof(float) * (size_t)N.np(), cudaMemcpyHostToDevice);
    cudaMemcpy(N.X, X, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice);
    forward(N, nullptr);
    cudaError_t e = cudaMemcpy(yhat, N.yh, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost);
    st = e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : cuda_status("cost-model forward");
    net_free(N);
    return st;
}

int openfft_mlp_loss_grad(int d, int hidden, const float* params, const float* X, const float* y, int n,
                          float* loss, float* grad)
{
    if (!params || !X || !y || !loss || !grad) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null pointer");
    int st = check_dims(d, hidden, n);
    if (st) return st;
    Net N;
    if ((st = net_alloc(N, d, hidden, n, true))) return st;
    cudaMemcpy(N.p, params, sizeof(float) * (size_t)N.np(), cudaMemcpyHostToDevice);
    cudaMemcpy(N.X, X, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice);
    cudaMemcpy(N.y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    forward(N, nullptr);
    backward(N, nullptr);
    cudaError_t e = cudaMemcpy(grad, N.g, sizeof(float) * (size_t)N.np(), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemcpy(loss, N.loss, sizeof(float), cudaMemcpyDeviceToHost);
    st = e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : cuda_status("cost-model backward");
    net_free(N);
    return st;
}

int openfft_mlp_train(int d, int hidden, const float* X, const float* y, int n, int steps, float lr,
                      float* params, float* losses)
{
    if (!params || !X || !y) return set_last_error(OPENFFT_ERR_INVALID_ARG, "null pointer");
    if (steps < 0) return set_last_error(OPENFFT_ERR_INVALID_ARG, "steps must be >= 0");
    int st = check_dims(d, hidden, n);
    if (st) return st;
    Net N;
    if ((st = net_alloc(N, d, hidden, n, true))) return st;
    const size_t np = (size_t)N.np();
    cudaMemcpy(N.p, params, sizeof(float) * np, cudaMemcpyHostToDevice);
    cudaMemcpy(N.X, X, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice);
    cudaMemcpy(N.y, y, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemset(N.m, 0, sizeof(float) * np);
    cudaMemset(N.v, 0, sizeof(float) * np);
    cudaMemset(N.t, 0, sizeof(int));
    std::vector<float> hl(losses ? (size_t)steps : 0);
    cudaStream_t s = nullptr;
    cudaGraphExec_t gx = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (!e) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            forward(N, s);
            backward(N, s);
            adam_step<<<blocks((int)np), kThreads, 0, s>>>(N.p, N.g, N.m, N.v, N.t, (int)np, lr, 0.9f, 0.999f, 1e-8f);
            advance_step<<<1, 1, 0, s>>>(N.t);
            e = cudaStreamEndCapture(s, &g);
        }
        if (!e) e = cudaGraphInstantiate(&gx, g, 0);
        if (g) cudaGraphDestroy(g);
    }
    for (int it = 0; it < steps && !e; ++it) {
        e = cudaGraphLaunch(gx, s);
        if (!e && losses) e = cudaMemcpyAsync(&hl[(size_t)it], N.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    }
    if (!e) e = cudaStreamSynchronize(s);
    if (!e) e = cudaMemcpy(params, N.p, sizeof(float) * np, cudaMemcpyDeviceToHost);
    if (!e && losses) std::memcpy(losses, hl.data(), sizeof(float) * hl.size());
    if (gx) cudaGraphExecDestroy(gx);
    if (s) cudaStreamDestroy(s);
    st = e ? set_last_error(OPENFFT_ERR_CUDA, cudaGetErrorString(e)) : OPENFFT_OK;
    net_free(N);
    return st;
}

}  // extern "C"
