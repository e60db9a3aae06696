// Learned step-time cost model: a small MLP trained and evaluated on the GPU
// with hand-written kernels (forward, backward, Adam).
//
// Network: x (n_in) -> relu(W1 x + b1) (h1) -> relu(W2 a1 + b2) (h2) -> W3 a2 + b3.
// Loss: mean over rows of (y - t)^2. Parameters live in one FP32 buffer in the
// order W1 [h1][n_in], b1 [h1], W2 [h2][h1], b2 [h2], W3 [h2], b3 [1].
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <memory>
#include <random>
#include <vector>

#include "plan.h"

namespace tn {

struct Mlp {
    int n_in = 0, h1 = 0, h2 = 0;
    int64_t n_params = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;  // params, grads, Adam moments
    int64_t adam_t = 0;
    // per-batch workspaces (grown on demand)
    int cap = 0;
    float *d_x = nullptr, *d_t = nullptr, *d_z1 = nullptr, *d_a1 = nullptr, *d_z2 = nullptr,
          *d_a2 = nullptr, *d_y = nullptr, *d_dy = nullptr, *d_dz2 = nullptr, *d_dz1 = nullptr;
    double *d_loss = nullptr;
    ~Mlp() {
        float *ps[] = {d_p, d_g, d_m, d_v, d_x, d_t, d_z1, d_a1, d_z2, d_a2, d_y, d_dy, d_dz2, d_dz1};
        for (float *p : ps)
            if (p) cudaFree(p);
        if (d_loss) cudaFree(d_loss);
    }
    int64_t off_w1() const { return 0; }
    int64_t off_b1() const { return (int64_t)h1 * n_in; }
    int64_t off_w2() const { return off_b1() + h1; }
    int64_t off_b2() const { return off_w2() + (int64_t)h2 * h1; }
    int64_t off_w3() const { return off_b2() + h2; }
    int64_t off_b3() const { return off_w3() + h2; }
};

// out[b][j] = act(sum_i in[b][i] * W[j][i] + bias[j]); z keeps the
// pre-activation when requested.
__global__ void mlp_dense_fwd(const float *__restrict__ in, const float *__restrict__ W,
                              const float *__restrict__ bias, float *__restrict__ z,
                              float *__restrict__ out, int rows, int n_in, int n_out, int relu) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * n_out) return;
    const int b = idx / n_out, j = idx % n_out;
    float acc = bias[j];
    for (int i = 0; i < n_in; ++i) acc = fmaf(in[(int64_t)b * n_in + i], W[(int64_t)j * n_in + i], acc);
    if (z) z[idx] = acc;
    out[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// dy = 2 (y - t) / rows, and the loss sum (FP64, one block reduction + atomics)
__global__ void mlp_loss_grad(const float *__restrict__ y, const float *__restrict__ t,
                              float *__restrict__ dy, double *loss, int rows) {
    __shared__ double sh[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < rows) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)rows;
        l = (double)d * (double)d / (double)rows;
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0]);
}

// dW[j][i] = sum_b dz[b][j] * in[b][i]; db[j] = sum_b dz[b][j]
__global__ void mlp_dense_wgrad(const float *__restrict__ dz, const float *__restrict__ in,
                                float *__restrict__ dW, float *__restrict__ db, int rows, int n_in,
                                int n_out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_out * (n_in + 1)) return;
    const int j = idx / (n_in + 1), i = idx % (n_in + 1);
    float acc = 0.f;
    if (i < n_in) {
        for (int b = 0; b < rows; ++b) acc = fmaf(dz[(int64_t)b * n_out + j], in[(int64_t)b * n_in + i], acc);
        dW[(int64_t)j * n_in + i] = acc;
    } else {
        for (int b = 0; b < rows; ++b) acc += dz[(int64_t)b * n_out + j];
        db[j] = acc;
    }
}

// dz_prev[b][i] = (sum_j dz[b][j] * W[j][i]) * relu'(z_prev[b][i])
__global__ void mlp_dense_bgrad(const float *__restrict__ dz, const float *__restrict__ W,
                                const float *__restrict__ z_prev, float *__restrict__ dz_prev,
                                int rows, int n_prev, int n_out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * n_prev) return;
    const int b = idx / n_prev, i = idx % n_prev;
    float acc = 0.f;
    for (int j = 0; j < n_out; ++j) acc = fmaf(dz[(int64_t)b * n_out + j], W[(int64_t)j * n_prev + i], acc);
    dz_prev[idx] = z_prev[idx] > 0.f ? acc : 0.f;
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void mlp_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                         float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

static void mlp_reserve(Mlp &m, int rows) {
    if (rows <= m.cap) return;
    float **ws[] = {&m.d_x, &m.d_t, &m.d_z1, &m.d_a1, &m.d_z2, &m.d_a2, &m.d_y, &m.d_dy, &m.d_dz2, &m.d_dz1};
    for (float **w : ws)
        if (*w) {
            cudaFree(*w);
            *w = nullptr;
        }
    const int width = std::max({m.n_in, m.h1, m.h2, 1});
    for (float **w : ws) TN_CUDA(cudaMalloc(w, sizeof(float) * (size_t)rows * width));
    if (!m.d_loss) TN_CUDA(cudaMalloc(&m.d_loss, sizeof(double)));
    m.cap = rows;
}

// Forward pass of rows already in d_x; result in d_y.
static void mlp_forward(Mlp &m, int rows, cudaStream_t st) {
    const float *P = m.d_p;
    mlp_dense_fwd<<<nblk((int64_t)rows * m.h1), 256, 0, st>>>(m.d_x, P + m.off_w1(), P + m.off_b1(),
                                                             m.d_z1, m.d_a1, rows, m.n_in, m.h1, 1);
    mlp_dense_fwd<<<nblk((int64_t)rows * m.h2), 256, 0, st>>>(m.d_a1, P + m.off_w2(), P + m.off_b2(),
                                                             m.d_z2, m.d_a2, rows, m.h1, m.h2, 1);
    mlp_dense_fwd<<<nblk(rows), 256, 0, st>>>(m.d_a2, P + m.off_w3(), P + m.off_b3(), nullptr, m.d_y,
                                              rows, m.h2, 1, 0);
    TN_CUDA(cudaGetLastError());
}

// Forward + backward of rows in d_x / d_t: loss into d_loss, gradient into d_g.
static void mlp_fwd_bwd(Mlp &m, int rows, cudaStream_t st) {
    mlp_forward(m, rows, st);
    TN_CUDA(cudaMemsetAsync(m.d_loss, 0, sizeof(double), st));
    mlp_loss_grad<<<nblk(rows), 256, 0, st>>>(m.d_y, m.d_t, m.d_dy, m.d_loss, rows);
    float *G = m.d_g;
    const float *P = m.d_p;
    // layer 3: dz3 = dy
    mlp_dense_wgrad<<<nblk((int64_t)(m.h2 + 1)), 256, 0, st>>>(m.d_dy, m.d_a2, G + m.off_w3(),
                                                              G + m.off_b3(), rows, m.h2, 1);
    mlp_dense_bgrad<<<nblk((int64_t)rows * m.h2), 256, 0, st>>>(m.d_dy, P + m.off_w3(), m.d_z2,
                                                               m.d_dz2, rows, m.h2, 1);
    // layer 2
    mlp_dense_wgrad<<<nblk((int64_t)m.h2 * (m.h1 + 1)), 256, 0, st>>>(m.d_dz2, m.d_a1, G + m.off_w2(),
                                                                     G + m.off_b2(), rows, m.h1, m.h2);
    mlp_dense_bgrad<<<nblk((int64_t)rows * m.h1), 256, 0, st>>>(m.d_dz2, P + m.off_w2(), m.d_z1,
                                                               m.d_dz1, rows, m.h1, m.h2);
    // layer 1
    mlp_dense_wgrad<<<nblk((int64_t)m.h1 * (m.n_in + 1)), 256, 0, st>>>(m.d_dz1, m.d_x, G + m.off_w1(),
                                                                       G + m.off_b1(), rows, m.n_in, m.h1);
    TN_CUDA(cudaGetLastError());
}

Mlp *mlp_create(int n_in, int h1, int h2, uint64_t seed) {
    if (n_in <= 0 || h1 <= 0 || h2 <= 0 || n_in > 4096 || h1 > 4096 || h2 > 4096)
        fail(TN_ERR_INVALID_ARG, "bad MLP sizes");
    auto m = std::make_unique<Mlp>();
    m->n_in = n_in;
    m->h1 = h1;
    m->h2 = h2;
    m->n_params = m->off_b3() + 1;
    // He initialisation for ReLU layers, zero biases
    std::vector<float> p((size_t)m->n_params, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan_in));
        for (int64_t i = 0; i < count; ++i) p[(size_t)(off + i)] = (float)nd(rng);
    };
    fill(m->off_w1(), (int64_t)h1 * n_in, n_in);
    fill(m->off_w2(), (int64_t)h2 * h1, h1);
    fill(m->off_w3(), h2, h2);
    const size_t bytes = sizeof(float) * (size_t)m->n_params;
    TN_CUDA(cudaMalloc(&m->d_p, bytes));
    TN_CUDA(cudaMalloc(&m->d_g, bytes));
    TN_CUDA(cudaMalloc(&m->d_m, bytes));
    TN_CUDA(cudaMalloc(&m->d_v, bytes));
    TN_CUDA(cudaMemcpy(m->d_p, p.data(), bytes, cudaMemcpyHostToDevice));
    TN_CUDA(cudaMemset(m->d_g, 0, bytes));
    TN_CUDA(cudaMemset(m->d_m, 0, bytes));
    TN_CUDA(cudaMemset(m->d_v, 0, bytes));
    return m.release();
}

void mlp_destroy(Mlp *m) { delete m; }
int64_t mlp_n_params(const Mlp &m) { return m.n_params; }

void mlp_set_params(Mlp &m, const float *p, int64_t n) {
    if (n != m.n_params) fail(TN_ERR_INVALID_ARG, "parameter count mismatch");
    TN_CUDA(cudaMemcpy(m.d_p, p, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice));
    TN_CUDA(cudaMemset(m.d_m, 0, sizeof(float) * (size_t)n));
    TN_CUDA(cudaMemset(m.d_v, 0, sizeof(float) * (size_t)n));
    m.adam_t = 0;
}

void mlp_get_params(const Mlp &m, float *p, int64_t n) {
    if (n != m.n_params) fail(TN_ERR_INVALID_ARG, "parameter count mismatch");
    TN_CUDA(cudaMemcpy(p, m.d_p, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost));
}

void mlp_loss_grad_host(Mlp &m, const float *X, const float *t, int rows, double *loss, float *grad) {
    if (rows <= 0) fail(TN_ERR_INVALID_ARG, "rows must be positive");
    mlp_reserve(m, rows);
    TN_CUDA(cudaMemcpy(m.d_x, X, sizeof(float) * (size_t)rows * m.n_in, cudaMemcpyHostToDevice));
    TN_CUDA(cudaMemcpy(m.d_t, t, sizeof(float) * (size_t)rows, cudaMemcpyHostToDevice));
    mlp_fwd_bwd(m, rows, nullptr);
    TN_CUDA(cudaMemcpy(loss, m.d_loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grad) TN_CUDA(cudaMemcpy(grad, m.d_g, sizeof(float) * (size_t)m.n_params, cudaMemcpyDeviceToHost));
}

// Mini-batch Adam over `epochs` passes of the rows (shuffled per epoch on the
// host; batches uploaded as they are used).
double mlp_train(Mlp &m, const float *X, const float *t, int rows, int epochs, int batch, float lr,
                 uint64_t seed) {
    if (rows <= 0 || epochs <= 0) fail(TN_ERR_INVALID_ARG, "rows and epochs must be positive");
    if (batch <= 0 || batch > rows) batch = rows;
    mlp_reserve(m, batch);
    std::vector<int> idx((size_t)rows);
    for (int i = 0; i < rows; ++i) idx[(size_t)i] = i;
    std::mt19937_64 rng(seed);
    std::vector<float> bx((size_t)batch * m.n_in), bt((size_t)batch);
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(idx.begin(), idx.end(), rng);
        double sum = 0.0;
        int nb = 0;
        for (int s = 0; s + batch <= rows; s += batch) {
            for (int r = 0; r < batch; ++r) {
                const int src = idx[(size_t)(s + r)];
                std::copy(X + (int64_t)src * m.n_in, X + (int64_t)(src + 1) * m.n_in,
                          bx.begin() + (int64_t)r * m.n_in);
                bt[(size_t)r] = t[src];
            }
            TN_CUDA(cudaMemcpy(m.d_x, bx.data(), sizeof(float) * bx.size(), cudaMemcpyHostToDevice));
            TN_CUDA(cudaMemcpy(m.d_t, bt.data(), sizeof(float) * bt.size(), cudaMemcpyHostToDevice));
            mlp_fwd_bwd(m, batch, nullptr);
            ++m.adam_t;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)m.adam_t), c2 = 1.f - std::pow(b2, (float)m.adam_t);
            mlp_adam<<<nblk(m.n_params), 256>>>(m.d_p, m.d_g, m.d_m, m.d_v, m.n_params, lr, b1, b2,
                                                1e-8f, c1, c2);
            TN_CUDA(cudaGetLastError());
            double l;
            TN_CUDA(cudaMemcpy(&l, m.d_loss, sizeof(double), cudaMemcpyDeviceToHost));
            sum += l;
            ++nb;
        }
        last = nb ? sum / nb : 0.0;
    }
    return last;
}

void mlp_predict(Mlp &m, const float *X, int rows, float *y) {
    if (rows <= 0) return;
    const int chunk = 1 << 16;
    for (int s = 0; s < rows; s += chunk) {
        const int r = std::min(chunk, rows - s);
        mlp_reserve(m, r);
        TN_CUDA(cudaMemcpy(m.d_x, X + (int64_t)s * m.n_in, sizeof(float) * (size_t)r * m.n_in,
                           cudaMemcpyHostToDevice));
        mlp_forward(m, r, nullptr);
        TN_CUDA(cudaMemcpy(y + s, m.d_y, sizeof(float) * (size_t)r, cudaMemcpyDeviceToHost));
    }
}

}  // namespace tn
