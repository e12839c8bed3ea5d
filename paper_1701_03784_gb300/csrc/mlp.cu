// Surrogate network ensemble: small multilayer perceptrons (tanh-GELU hidden layers, linear
// output) that map sweep parameters to simulation outputs, trained and evaluated on the
// GPU by the kernels in this file (FP32 on CUDA cores) and k_mlp_tc.cu (BF16 tensor-core
// inference, and optionally the training products: pic_mlp_set_training).  The paper has
// no counterpart.
//
// Layout: per member, the layers' parameters one after another, W_l (n_out x n_in,
// row-major) then b_l; members follow each other at a fixed stride.  Activations are
// row-major (sample x unit) per member.  Minibatch indices come from a counter-based hash
// of (seed, member, step, row), so a training run is reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pic_internal.h"

namespace pic {

namespace {
constexpr int GT = 16;           // GEMM tile
constexpr float C_GELU = 0.7978845608028654f;   // sqrt(2/pi)

// C(z)[m][n] (+)= sum_k A(z, m, k) B(z, k, n), operands addressed by strides; z = member
struct GemmArgs {
    const float *A, *B;
    float *C;
    int M, N, K;
    long long sAz, sBz, sCz;
    int sAm, sAk, sBk, sBn, ldc;
    int accumulate;
};

__global__ void __launch_bounds__(GT * GT) k_gemm(GemmArgs g) {
    __shared__ float As[GT][GT + 1], Bs[GT][GT + 1];
    const int z = blockIdx.z;
    const float *A = g.A + z * g.sAz, *B = g.B + z * g.sBz;
    float *C = g.C + z * g.sCz;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * GT + ty, n = blockIdx.x * GT + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < g.K; k0 += GT) {
        const int ka = k0 + tx, kb = k0 + ty;
        const int ma = blockIdx.y * GT + ty;
        As[ty][tx] = (ma < g.M && ka < g.K) ? A[(long long)ma * g.sAm + (long long)ka * g.sAk] : 0.f;
        Bs[ty][tx] = (kb < g.K && n < g.N) ? B[(long long)kb * g.sBk + (long long)n * g.sBn] : 0.f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GT; kk++) acc = fmaf(As[ty][kk], Bs[kk][tx], acc);
        __syncthreads();
    }
    if (m < g.M && n < g.N) {
        float *c = C + (long long)m * g.ldc + n;
        *c = g.accumulate ? *c + acc : acc;
    }
}

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.f + tanhf(C_GELU * (z + 0.044715f * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
    const float t = tanhf(C_GELU * (z + 0.044715f * z * z * z));
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * C_GELU * (1.f + 3.f * 0.044715f * z * z);
}

// Z += b (per column); A = gelu(Z) for hidden layers, A = Z for the output layer
__global__ void k_bias_act(float *Z, float *A, const float *b, long long bz, int rows, int cols,
                           long long sz, int act) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (i >= (long long)rows * cols) return;
    const float v = Z[z * sz + i] + b[z * bz + (int)(i % cols)];
    Z[z * sz + i] = v;
    if (A) A[z * sz + i] = act ? gelu(v) : v;
}

// G = scale (Y - T); loss[z] += sum (Y - T)^2 / count
__global__ void k_loss_grad(const float *Y, const float *T, float *G, long long n, long long sY,
                            long long sT, long long sG, float scale, float *loss) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    float e = 0.f;
    if (i < n) {
        e = Y[z * sY + i] - T[z * sT + i];
        G[z * sG + i] = scale * e;
    }
    float s = e * e;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (loss && (threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(loss + z, s / (float)n);
}

__global__ void k_gelu_back(float *G, const float *Z, long long n, long long sG, long long sZ) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) G[blockIdx.y * sG + i] *= gelu_grad(Z[blockIdx.y * sZ + i]);
}

// db[j] = sum_i G[i][j]
__global__ void k_colsum(const float *G, float *db, int rows, int cols, long long sg, long long sb) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; i++) s += G[z * sg + (long long)i * cols + j];
    db[z * sb + j] = s;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    // splitmix64 finaliser
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// `rows` samples per member into the member's batch buffers (row stride mrows): drawn from
// n with replacement (random = 1) or rows 0.. of X and T (random = 0)
__global__ void k_gather(const float *X, const float *T, float *Xb, float *Tb, long long n, int rows,
                         int mrows, int din, int dout, unsigned long long seed, long long step,
                         int random) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (r >= rows) return;
    long long s = r;
    if (random) {
        const unsigned long long h = mix64(
            seed ^ mix64(((unsigned long long)z << 48) ^ ((unsigned long long)step << 20) ^ r));
        s = (long long)(h % (unsigned long long)n);
    }
    const long long o = (long long)z * mrows + r;
    for (int k = 0; k < din; k++) Xb[o * din + k] = X[s * din + k];
    for (int k = 0; k < dout; k++) Tb[o * dout + k] = T[s * dout + k];
}

// rows of each member's output batch into Y (members x n x dout) at row offset c0
__global__ void k_copy_out(const float *A, float *Y, int rows, int dout, int mrows, long long n,
                           long long c0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (i >= (long long)rows * dout) return;
    Y[((long long)z * n + c0) * dout + i] = A[(long long)z * mrows * dout + i];
}

__global__ void k_to_f32(const double *src, float *dst, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

inline unsigned blocks(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }
}  // namespace


struct MlpImpl {
    int device = 0;
    Allocator al;
    std::vector<void *> allocs;
    int E = 0, L = 0, max_batch = 0, maxw = 0;
    std::vector<int> sz;
    std::vector<long long> woff, boff;
    long long P = 0;
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr, *Tb = nullptr,
          *loss = nullptr;
    double *stage = nullptr;
    std::vector<float *> act, pre;
    float *gbuf[2] = {nullptr, nullptr};
    long long adam_step = 0;
    MlpTc tc;               // BF16 tensor-core copy of the parameters
    bool tc_dirty = true;   // parameters changed since it was packed
    // training products on the tensor cores (pic_mlp_set_training): packed BF16 operand
    // scratch and the bounded-wait counter
    bool train_tc = false, gemm_tc = false;
    uint16_t *tsa = nullptr, *tsb = nullptr;
    unsigned int *terr = nullptr;

    ~MlpImpl() {
        cudaSetDevice(device);
        cudaDeviceSynchronize();
        for (void *p : allocs) {
            if (al.free) al.free(p, al.ctx);
            else cudaFree(p);
        }
    }
    template <class T>
    pic_status dalloc(T *&p, long long n) {
        const size_t bytes = sizeof(T) * (size_t)std::max<long long>(n, 1);
        void *v = nullptr;
        if (al.alloc) v = al.alloc(bytes, al.ctx);
        else if (cudaMalloc(&v, bytes) != cudaSuccess) v = nullptr;
        if (!v) {
            set_error("pic_mlp_create: device allocation of %zu bytes failed", bytes);
            return PIC_ERR_OOM;
        }
        allocs.push_back(v);
        p = static_cast<T *>(v);
        return PIC_OK;
    }

    pic_status init(int members, int layers, const int32_t *sizes, int batch) {
        E = members;
        L = layers;
        max_batch = batch;
        sz.assign(sizes, sizes + layers + 1);
        maxw = *std::max_element(sz.begin(), sz.end());
        for (int l = 0; l < L; l++) {
            woff.push_back(P);
            P += (long long)sz[l + 1] * sz[l];
            boff.push_back(P);
            P += sz[l + 1];
        }
        pic_status st;
        if ((st = dalloc(params, E * P)) || (st = dalloc(grads, E * P)) || (st = dalloc(am, E * P)) ||
            (st = dalloc(av, E * P)) || (st = dalloc(stage, E * P)) ||
            (st = dalloc(Tb, (long long)E * batch * sz[L])) || (st = dalloc(loss, E)) ||
            (st = dalloc(gbuf[0], (long long)E * batch * maxw)) ||
            (st = dalloc(gbuf[1], (long long)E * batch * maxw)))
            return st;
        act.assign(L + 1, nullptr);
        pre.assign(L, nullptr);
        for (int l = 0; l <= L; l++)
            if ((st = dalloc(act[l], (long long)E * batch * sz[l]))) return st;
        for (int l = 0; l < L; l++)
            if ((st = dalloc(pre[l], (long long)E * batch * sz[l + 1]))) return st;
        // tensor-core inference: every width at most 256
        tc.ok = L <= MLP_MAX_LAYERS && maxw <= 256;
        if (tc.ok) {
            tc.E = E;
            tc.L = L;
            for (int l = 0; l < L; l++) {
                tc.k[l] = sz[l];
                tc.n[l] = sz[l + 1];
                tc.kp[l] = (sz[l] + 15) / 16 * 16;
                tc.np[l] = (sz[l + 1] + 15) / 16 * 16;
                tc.woff[l] = tc.wmember;
                tc.wmember += (long long)tc.kp[l] * tc.np[l];
                tc.boff[l] = tc.bmember;
                tc.bmember += tc.np[l];
            }
            if ((st = dalloc(tc.w, E * tc.wmember)) || (st = dalloc(tc.b, E * tc.bmember)) ||
                (st = dalloc(tc.err, 1)))
                return st;
            const long long mp = (std::max(max_batch, maxw) + 127) / 128 * 128;
            if ((st = dalloc(tsa, (long long)E * mp * 256)) ||
                (st = dalloc(tsb, (long long)E * 256 * 256)) || (st = dalloc(terr, 1)))
                return st;
            PIC_CUDA_TRY(cudaMemset(terr, 0, sizeof(unsigned int)));
        }
        PIC_CUDA_TRY(cudaMemset(params, 0, sizeof(float) * E * P));
        PIC_CUDA_TRY(cudaMemset(am, 0, sizeof(float) * E * P));
        PIC_CUDA_TRY(cudaMemset(av, 0, sizeof(float) * E * P));
        return PIC_OK;
    }

    // timeouts of the training products since the last check (synchronises when the
    // tensor-core products were on)
    pic_status tc_errors(const char *who, cudaStream_t s) {
        if (!train_tc || !terr) return PIC_OK;
        unsigned int e = 0;
        PIC_CUDA_TRY(cudaMemcpyAsync(&e, terr, sizeof e, cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        if (e) {
            PIC_CUDA_TRY(cudaMemsetAsync(terr, 0, sizeof e, s));
            set_error("%s: %u tensor-core waits timed out", who, e);
            return PIC_ERR_TIMEOUT;
        }
        return PIC_OK;
    }

    void gemm(const GemmArgs &g, cudaStream_t s) {
        if (gemm_tc) {
            const TcGemmOp op{g.A, g.B, g.C, g.M, g.N, g.K, g.sAz, g.sBz, g.sCz,
                              g.sAm, g.sAk, g.sBk, g.sBn, g.ldc, g.accumulate};
            if (mlp_tc_gemm(op, E, tsa, tsb, terr, s)) return;
        }
        dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, E);
        k_gemm<<<grid, dim3(GT, GT), 0, s>>>(g);
        PIC_LAUNCHED();
    }

    // all layers for `rows` samples; the input of member z is X0 + z * sX0z (row-major)
    void forward(int rows, const float *X0, long long sX0z, cudaStream_t s) {
        const float *A = X0;
        long long sAz = sX0z;
        for (int l = 0; l < L; l++) {
            const int K = sz[l], N = sz[l + 1];
            GemmArgs g{A, params + woff[l], pre[l], rows, N, K, sAz, P,
                       (long long)max_batch * N, K, 1, 1, K, N, 0};
            gemm(g, s);
            k_bias_act<<<dim3(blocks((long long)rows * N), E), 256, 0, s>>>(
                pre[l], act[l + 1], params + boff[l], P, rows, N, (long long)max_batch * N,
                l < L - 1);
            PIC_LAUNCHED();
            A = act[l + 1];
            sAz = (long long)max_batch * N;
        }
    }

    // gradients of the mean squared error of act[L] against Tb (rows samples), inputs act[0]
    void backward(int rows, float *loss_out, cudaStream_t s) {
        const int dout = sz[L];
        float *G = gbuf[0], *Gn = gbuf[1];
        const long long sg = (long long)max_batch * maxw;
        k_loss_grad<<<dim3(blocks((long long)rows * dout), E), 256, 0, s>>>(
            act[L], Tb, G, (long long)rows * dout, (long long)max_batch * dout,
            (long long)max_batch * dout, sg, 2.f / (float)((long long)rows * dout), loss_out);
        PIC_LAUNCHED();
        // G is stored with the layer's width as row stride, member stride sg
        for (int l = L - 1; l >= 0; l--) {
            const int K = sz[l], N = sz[l + 1];
            if (l < L - 1)
                k_gelu_back<<<dim3(blocks((long long)rows * N), E), 256, 0, s>>>(
                    G, pre[l], (long long)rows * N, sg, (long long)max_batch * N);
                PIC_LAUNCHED();
            GemmArgs dw{G, act[l], grads + woff[l], N, K, rows, sg, (long long)max_batch * K, P,
                        1, N, K, 1, K, 0};
            gemm(dw, s);
            k_colsum<<<dim3(blocks(N), E), 256, 0, s>>>(G, grads + boff[l], rows, N, sg, P);
            PIC_LAUNCHED();
            if (l > 0) {
                GemmArgs dx{G, params + woff[l], Gn, rows, K, N, sg, P, sg, N, 1, K, 1, K, 0};
                gemm(dx, s);
                std::swap(G, Gn);
            }
        }
    }
};

}  // namespace pic

using namespace pic;

struct pic_mlp {
    MlpImpl *impl = nullptr;
    ~pic_mlp() { delete impl; }
};

#define MLP_CHECK(m, name)                                   \
    do {                                                     \
        if (!(m) || !(m)->impl) {                            \
            pic::set_error("%s: null network", name);        \
            return PIC_ERR_ARG;                              \
        }                                                    \
        cudaError_t e__ = cudaSetDevice((m)->impl->device);  \
        if (e__ != cudaSuccess) {                            \
            pic::set_error("%s: %s", name, cudaGetErrorString(e__)); \
            return PIC_ERR_CUDA;                             \
        }                                                    \
    } while (0)

extern "C" pic_status pic_mlp_create(int32_t n_members, int32_t n_layers, const int32_t *sizes,
                                     int32_t max_batch, pic_mlp **out) try {
    if (!sizes || !out || n_members < 1 || n_members > 64 || n_layers < 1 || n_layers > 16 ||
        max_batch < 1 || max_batch > (1 << 20)) {
        set_error("pic_mlp_create: bad arguments");
        return PIC_ERR_ARG;
    }
    for (int l = 0; l <= n_layers; l++)
        if (sizes[l] < 1 || sizes[l] > 4096) {
            set_error("pic_mlp_create: layer width %d out of range", sizes[l]);
            return PIC_ERR_ARG;
        }
    std::unique_ptr<pic_mlp> m(new (std::nothrow) pic_mlp);
    if (!m || !(m->impl = new (std::nothrow) MlpImpl)) {
        set_error("pic_mlp_create: out of host memory");
        return PIC_ERR_OOM;
    }
    PIC_CUDA_TRY(cudaGetDevice(&m->impl->device));
    m->impl->al = current_allocator();
    pic_status st = m->impl->init(n_members, n_layers, sizes, max_batch);
    if (st != PIC_OK) return st;
    *out = m.release();
    return PIC_OK;
}
PIC_CATCH("pic_mlp_create")

extern "C" pic_status pic_mlp_param_count(pic_mlp *m, int64_t *per_member) try {
    MLP_CHECK(m, "pic_mlp_param_count");
    if (!per_member) {
        set_error("pic_mlp_param_count: null output");
        return PIC_ERR_ARG;
    }
    *per_member = m->impl->P;
    return PIC_OK;
}
PIC_CATCH("pic_mlp_param_count")

extern "C" pic_status pic_mlp_params_set(pic_mlp *m, const double *params) try {
    MLP_CHECK(m, "pic_mlp_params_set");
    MlpImpl &x = *m->impl;
    if (!params) {
        set_error("pic_mlp_params_set: null parameters");
        return PIC_ERR_ARG;
    }
    const long long n = x.E * x.P;
    PIC_CUDA_TRY(cudaMemcpy(x.stage, params, sizeof(double) * n, cudaMemcpyHostToDevice));
    k_to_f32<<<blocks(n), 256>>>(x.stage, x.params, n);
    PIC_LAUNCHED();
    PIC_CUDA_TRY(cudaMemset(x.am, 0, sizeof(float) * n));
    PIC_CUDA_TRY(cudaMemset(x.av, 0, sizeof(float) * n));
    x.adam_step = 0;
    x.tc_dirty = true;
    PIC_CUDA_TRY(cudaDeviceSynchronize());
    return PIC_OK;
}
PIC_CATCH("pic_mlp_params_set")

extern "C" pic_status pic_mlp_params_get(pic_mlp *m, double *params) try {
    MLP_CHECK(m, "pic_mlp_params_get");
    MlpImpl &x = *m->impl;
    if (!params) {
        set_error("pic_mlp_params_get: null output");
        return PIC_ERR_ARG;
    }
    std::vector<float> h(x.E * x.P);
    PIC_CUDA_TRY(cudaDeviceSynchronize());
    PIC_CUDA_TRY(cudaMemcpy(h.data(), x.params, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); i++) params[i] = h[i];
    return PIC_OK;
}
PIC_CATCH("pic_mlp_params_get")

extern "C" pic_status pic_mlp_grad(pic_mlp *m, const float *X, const float *T, int64_t n,
                                   double *grads, double *loss, void *st) try {
    MLP_CHECK(m, "pic_mlp_grad");
    MlpImpl &x = *m->impl;
    if (!X || !T || !grads || n < 1 || n > x.max_batch) {
        set_error("pic_mlp_grad: bad arguments (n must be 1..max_batch)");
        return PIC_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)st;
    const int rows = (int)n;
    k_gather<<<dim3(blocks(rows), x.E), 256, 0, s>>>(X, T, x.act[0], x.Tb, n, rows, x.max_batch,
                                                     x.sz[0], x.sz[x.L], 0, 0, 0);
    PIC_LAUNCHED();
    PIC_CUDA_TRY(cudaMemsetAsync(x.loss, 0, sizeof(float) * x.E, s));
    x.gemm_tc = x.train_tc;
    x.forward(rows, x.act[0], (long long)x.max_batch * x.sz[0], s);
    x.backward(rows, x.loss, s);
    x.gemm_tc = false;
    pic_status ts = x.tc_errors("pic_mlp_grad", s);
    if (ts != PIC_OK) return ts;
    std::vector<float> h(x.E * x.P), hl(x.E);
    PIC_CUDA_TRY(cudaMemcpyAsync(h.data(), x.grads, sizeof(float) * h.size(),
                                 cudaMemcpyDeviceToHost, s));
    PIC_CUDA_TRY(cudaMemcpyAsync(hl.data(), x.loss, sizeof(float) * x.E, cudaMemcpyDeviceToHost, s));
    PIC_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t i = 0; i < h.size(); i++) grads[i] = h[i];
    if (loss)
        for (int z = 0; z < x.E; z++) loss[z] = hl[z];
    return PIC_OK;
}
PIC_CATCH("pic_mlp_grad")

extern "C" pic_status pic_mlp_train(pic_mlp *m, const float *X, const float *T, int64_t n,
                                    int32_t batch, int64_t steps, double lr, uint64_t seed,
                                    double *last_loss, void *st) try {
    MLP_CHECK(m, "pic_mlp_train");
    MlpImpl &x = *m->impl;
    if (!X || !T || n < 1 || batch < 1 || batch > x.max_batch || steps < 0 || !(lr > 0)) {
        set_error("pic_mlp_train: bad arguments (batch must be 1..max_batch)");
        return PIC_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)st;
    const long long np = x.E * x.P;
    x.tc_dirty = true;
    x.gemm_tc = x.train_tc;
    for (long long k = 0; k < steps; k++) {
        k_gather<<<dim3(blocks(batch), x.E), 256, 0, s>>>(X, T, x.act[0], x.Tb, n, batch,
                                                          x.max_batch, x.sz[0], x.sz[x.L], seed,
                                                          x.adam_step, 1);
        PIC_LAUNCHED();
        const bool last = k == steps - 1;
        if (last) PIC_CUDA_TRY(cudaMemsetAsync(x.loss, 0, sizeof(float) * x.E, s));
        x.forward(batch, x.act[0], (long long)x.max_batch * x.sz[0], s);
        x.backward(batch, last ? x.loss : nullptr, s);
        x.adam_step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)x.adam_step);
        const float c2 = 1.f - std::pow(b2, (float)x.adam_step);
        k_adam<<<blocks(np), 256, 0, s>>>(x.params, x.grads, x.am, x.av, np, (float)lr, b1, b2,
                                          1e-8f, c1, c2);
        PIC_LAUNCHED();
    }
    x.gemm_tc = false;
    PIC_CUDA_TRY(cudaGetLastError());
    pic_status ts = x.tc_errors("pic_mlp_train", s);
    if (ts != PIC_OK) return ts;
    if (last_loss) {
        std::vector<float> hl(x.E, 0.f);
        if (steps > 0)
            PIC_CUDA_TRY(cudaMemcpyAsync(hl.data(), x.loss, sizeof(float) * x.E,
                                         cudaMemcpyDeviceToHost, s));
        PIC_CUDA_TRY(cudaStreamSynchronize(s));
        for (int z = 0; z < x.E; z++) last_loss[z] = hl[z];
    }
    return PIC_OK;
}
PIC_CATCH("pic_mlp_train")

extern "C" pic_status pic_mlp_forward(pic_mlp *m, const float *X, float *Y, int64_t n,
                                      int32_t tensor_cores, void *st) try {
    MLP_CHECK(m, "pic_mlp_forward");
    MlpImpl &x = *m->impl;
    if (!X || !Y || n < 0) {
        set_error("pic_mlp_forward: bad arguments");
        return PIC_ERR_ARG;
    }
    if (tensor_cores) {
        if (!x.tc.ok) {
            set_error("pic_mlp_forward: the tensor-core path needs layer widths of at most 256");
            return PIC_ERR_ARG;
        }
        if (x.tc_dirty) {
            mlp_tc_pack(x.tc, x.params, x.P, x.woff.data(), x.boff.data(), (cudaStream_t)st);
            x.tc_dirty = false;
        }
        return mlp_tc_forward(x.tc, X, Y, n, (cudaStream_t)st);
    }
    cudaStream_t s = (cudaStream_t)st;
    const int din = x.sz[0], dout = x.sz[x.L];
    for (long long c0 = 0; c0 < n; c0 += x.max_batch) {
        const int rows = (int)std::min<long long>(x.max_batch, n - c0);
        x.forward(rows, X + c0 * din, 0, s);
        k_copy_out<<<dim3(blocks((long long)rows * dout), x.E), 256, 0, s>>>(
            x.act[x.L], Y, rows, dout, x.max_batch, n, c0);
        PIC_LAUNCHED();
    }
    PIC_CUDA_TRY(cudaGetLastError());
    return PIC_OK;
}
PIC_CATCH("pic_mlp_forward")

extern "C" pic_status pic_mlp_set_training(pic_mlp *m, int32_t tensor_cores) try {
    MLP_CHECK(m, "pic_mlp_set_training");
    MlpImpl &x = *m->impl;
    if (tensor_cores && !x.tc.ok) {
        set_error("pic_mlp_set_training: tensor-core products need widths of at most 256");
        return PIC_ERR_ARG;
    }
    x.train_tc = tensor_cores != 0;
    return PIC_OK;
}
PIC_CATCH("pic_mlp_set_training")

extern "C" pic_status pic_mlp_set_wait_limit(pic_mlp *m, int64_t polls) try {
    MLP_CHECK(m, "pic_mlp_set_wait_limit");
    if (polls < 0) {
        set_error("pic_mlp_set_wait_limit: negative poll count");
        return PIC_ERR_ARG;
    }
    m->impl->tc.wait_polls = polls;
    return PIC_OK;
}
PIC_CATCH("pic_mlp_set_wait_limit")

extern "C" void pic_mlp_destroy(pic_mlp *m) { delete m; }
