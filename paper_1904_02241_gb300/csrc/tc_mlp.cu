// Learned cost model: a small FP32 multi-layer perceptron with its own forward, backward and
// Adam kernels, and the graph/subgraph feature extractor that feeds it.  The network picks the
// TOCAB block count, the load-balancing variant and the push/pull direction (the trade-offs of
// Sec. 3.1 block size, Sec. 3.2 load balancing, Sec. 4.3 sensitivity); it never changes results.
//   z = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3, heads = softmax slices of z,
//   loss = mean over samples of the summed cross-entropy of the heads.
// Every reduction over samples runs in a fixed order (one thread per weight), so training is
// deterministic.
#include "tc_common_dev.cuh"

struct tc_mlp {
    int32_t nin = 16, nhid = 64, nheads = 0, nout = 0;
    int32_t head_sizes[8] = {0};
    int64_t nparams = 0;
    int64_t step = 0;
    tc::DevBuf params, grads, adam_m, adam_v;
    tc::DevBuf work;      // activations of the current batch
    tc::DevBuf flag;      // int: set by the label check
    int32_t work_n = 0;
};

namespace tc {

struct MlpOff {
    int64_t W1, b1, W2, b2, W3, b3, total;
};

static MlpOff mlp_offsets(const tc_mlp *m) {
    MlpOff o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)m->nin * m->nhid;
    o.W2 = o.b1 + m->nhid;
    o.b2 = o.W2 + (int64_t)m->nhid * m->nhid;
    o.W3 = o.b2 + m->nhid;
    o.b3 = o.W3 + (int64_t)m->nhid * m->nout;
    o.total = o.b3 + m->nout;
    return o;
}

// A[n,o] = b[o] + sum_i X[n,i] W[i,o];  H = relu(A) (H may be null)
__global__ void k_dense_fwd(const float *X, const float *W, const float *b, float *A, float *H, int32_t N, int32_t I,
                            int32_t O) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * O) return;
    const int32_t n = (int32_t)(t / O), o = (int32_t)(t % O);
    float acc = b[o];
    for (int32_t i = 0; i < I; ++i) acc += X[(int64_t)n * I + i] * W[(int64_t)i * O + o];
    A[t] = acc;
    if (H) H[t] = acc > 0.0f ? acc : 0.0f;
}

struct Heads {
    int32_t n;
    int32_t size[8];
};

// *bad = 1 when some label lies outside [0, size of its head); checked before any kernel
// indexes the logits with a label.
__global__ void k_check_labels(const int32_t *Y, int32_t N, Heads h, int *bad) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * h.n) return;
    const int32_t k = (int32_t)(t % h.n);
    const int32_t y = Y[t];
    if (y < 0 || y >= h.size[k]) *bad = 1;
}

// per sample: cross-entropy of every head, dZ = (softmax - onehot) / N
__global__ void k_softmax_ce(const float *Z, const int32_t *Y, int32_t N, int32_t O, Heads h, float *dZ,
                             double *loss_per_sample) {
    const int32_t n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double loss = 0.0;
    int32_t off = 0;
    for (int32_t k = 0; k < h.n; ++k) {
        const float *z = Z + (int64_t)n * O + off;
        const int32_t c = h.size[k];
        float mx = z[0];
        for (int32_t i = 1; i < c; ++i) mx = fmaxf(mx, z[i]);
        float se = 0.0f;
        for (int32_t i = 0; i < c; ++i) se += expf(z[i] - mx);
        const float lse = mx + logf(se);
        const int32_t y = Y[(int64_t)n * h.n + k];
        loss += (double)(lse - z[y]);
        if (dZ)
            for (int32_t i = 0; i < c; ++i)
                dZ[(int64_t)n * O + off + i] = (expf(z[i] - lse) - (i == y ? 1.0f : 0.0f)) / (float)N;
        off += c;
    }
    loss_per_sample[n] = loss;
}

// dW[i,o] = sum_n Xin[n,i] dA[n,o]; db[o] = sum_n dA[n,o]  (one thread per weight, n in order)
__global__ void k_dense_bwd_w(const float *Xin, const float *dA, float *dW, float *db, int32_t N, int32_t I, int32_t O) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < (int64_t)I * O) {
        const int32_t i = (int32_t)(t / O), o = (int32_t)(t % O);
        float acc = 0.0f;
        for (int32_t n = 0; n < N; ++n) acc += Xin[(int64_t)n * I + i] * dA[(int64_t)n * O + o];
        dW[t] = acc;
    } else if (t < (int64_t)I * O + O) {
        const int32_t o = (int32_t)(t - (int64_t)I * O);
        float acc = 0.0f;
        for (int32_t n = 0; n < N; ++n) acc += dA[(int64_t)n * O + o];
        db[o] = acc;
    }
}

// dAin[n,i] = (sum_o dA[n,o] W[i,o]) * (Ain[n,i] > 0)
__global__ void k_dense_bwd_x(const float *dA, const float *W, const float *Ain, float *dAin, int32_t N, int32_t I,
                              int32_t O) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)N * I) return;
    const int32_t n = (int32_t)(t / I), i = (int32_t)(t % I);
    float acc = 0.0f;
    for (int32_t o = 0; o < O; ++o) acc += dA[(int64_t)n * O + o] * W[(int64_t)i * O + o];
    dAin[t] = Ain[t] > 0.0f ? acc : 0.0f;
}

// Adam (Kingma & Ba 2015, Algorithm 1), bias-corrected
__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t P, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= P) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.0f - b1) * gt;
    const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    const float mh = mt / c1, vh = vt / c2;
    p[t] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_sum_ordered(const double *x, int32_t n, double *out) {
    __shared__ double red[32];
    double t = 0.0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) t += x[i];
    t = block_sum<double>(t, red);
    if (threadIdx.x == 0) *out = t;
}

static int grid_for(int64_t n) { return (int)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

// workspace: X, A1, H1, A2, H2, Z, dZ, dA2, dA1 (floats), Y (ints), loss (doubles)
struct MlpWork {
    float *X, *A1, *H1, *A2, *H2, *Z, *dZ, *dA2, *dA1;
    int32_t *Y;
    double *loss, *loss_sum;
};

static int mlp_work(tc_mlp *m, int32_t N, MlpWork *w) {
    const int64_t f = (int64_t)N * (m->nin + 4 * m->nhid + 2 * m->nout + 2 * m->nhid) + 64;
    const int64_t bytes = f * 4 + (int64_t)N * m->nheads * 4 + (int64_t)(N + 2) * 8 + 1024;
    TC_TRY(m->work.alloc((size_t)bytes));
    char *p = m->work.as<char>();
    auto take = [&](int64_t nbytes) {
        char *q = p;
        p += (nbytes + 255) / 256 * 256;
        return q;
    };
    w->loss = reinterpret_cast<double *>(take((int64_t)(N + 1) * 8));
    w->loss_sum = reinterpret_cast<double *>(take(8));
    w->X = reinterpret_cast<float *>(take((int64_t)N * m->nin * 4));
    w->A1 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->H1 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->A2 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->H2 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->Z = reinterpret_cast<float *>(take((int64_t)N * m->nout * 4));
    w->dZ = reinterpret_cast<float *>(take((int64_t)N * m->nout * 4));
    w->dA2 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->dA1 = reinterpret_cast<float *>(take((int64_t)N * m->nhid * 4));
    w->Y = reinterpret_cast<int32_t *>(take((int64_t)N * m->nheads * 4));
    if (p > m->work.as<char>() + m->work.bytes) return fail(TC_ERR_OOM, "mlp workspace layout overflow");
    return TC_OK;
}

static int mlp_forward_dev(tc_mlp *m, const MlpWork &w, int32_t N, cudaStream_t s) {
    const MlpOff o = mlp_offsets(m);
    const float *P = m->params.as<float>();
    k_dense_fwd<<<grid_for((int64_t)N * m->nhid), 256, 0, s>>>(w.X, P + o.W1, P + o.b1, w.A1, w.H1, N, m->nin, m->nhid);
    k_dense_fwd<<<grid_for((int64_t)N * m->nhid), 256, 0, s>>>(w.H1, P + o.W2, P + o.b2, w.A2, w.H2, N, m->nhid, m->nhid);
    k_dense_fwd<<<grid_for((int64_t)N * m->nout), 256, 0, s>>>(w.H2, P + o.W3, P + o.b3, w.Z, nullptr, N, m->nhid, m->nout);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

static Heads heads_of(const tc_mlp *m) {
    Heads h;
    h.n = m->nheads;
    for (int k = 0; k < 8; ++k) h.size[k] = k < m->nheads ? m->head_sizes[k] : 0;
    return h;
}

static int mlp_loss_grad_dev(tc_mlp *m, const MlpWork &w, int32_t N, bool want_grad, cudaStream_t s) {
    const MlpOff o = mlp_offsets(m);
    const float *P = m->params.as<float>();
    float *G = m->grads.as<float>();
    TC_TRY(mlp_forward_dev(m, w, N, s));
    k_softmax_ce<<<grid_for(N), 256, 0, s>>>(w.Z, w.Y, N, m->nout, heads_of(m), want_grad ? w.dZ : nullptr, w.loss);
    k_sum_ordered<<<1, 256, 0, s>>>(w.loss, N, w.loss_sum);
    TC_LAUNCH_CHECK();
    if (!want_grad) return TC_OK;
    k_dense_bwd_w<<<grid_for((int64_t)m->nhid * m->nout + m->nout), 256, 0, s>>>(w.H2, w.dZ, G + o.W3, G + o.b3, N, m->nhid,
                                                                                m->nout);
    k_dense_bwd_x<<<grid_for((int64_t)N * m->nhid), 256, 0, s>>>(w.dZ, P + o.W3, w.A2, w.dA2, N, m->nhid, m->nout);
    k_dense_bwd_w<<<grid_for((int64_t)m->nhid * m->nhid + m->nhid), 256, 0, s>>>(w.H1, w.dA2, G + o.W2, G + o.b2, N, m->nhid,
                                                                                m->nhid);
    k_dense_bwd_x<<<grid_for((int64_t)N * m->nhid), 256, 0, s>>>(w.dA2, P + o.W2, w.A1, w.dA1, N, m->nhid, m->nhid);
    k_dense_bwd_w<<<grid_for((int64_t)m->nin * m->nhid + m->nhid), 256, 0, s>>>(w.X, w.dA1, G + o.W1, G + o.b1, N, m->nin,
                                                                               m->nhid);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

static int copy_to_dev(void *dst, const void *src, size_t bytes, int mem, cudaStream_t s) {
    TC_CUDA(cudaMemcpyAsync(dst, src, bytes, mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return TC_OK;
}

// Every label of Y (device, N x nheads) inside its head, else TC_ERR_INVALID_ARG.
static int check_labels(tc_mlp *m, const int32_t *Y, int32_t N, cudaStream_t s) {
    TC_TRY(m->flag.alloc(16));
    TC_CUDA(cudaMemsetAsync(m->flag.p, 0, 4, s));
    k_check_labels<<<grid_for((int64_t)N * m->nheads), 256, 0, s>>>(Y, N, heads_of(m), m->flag.as<int>());
    TC_LAUNCH_CHECK();
    int bad = 0;
    TC_CUDA(cudaMemcpyAsync(&bad, m->flag.p, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (bad) return fail(TC_ERR_INVALID_ARG, "mlp: a label lies outside [0, size of its head)");
    return TC_OK;
}

static int adam_dev(tc_mlp *m, float lr, float b1, float b2, float eps, cudaStream_t s) {
    m->step += 1;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    k_adam<<<grid_for(m->nparams), 256, 0, s>>>(m->params.as<float>(), m->grads.as<float>(), m->adam_m.as<float>(),
                                               m->adam_v.as<float>(), m->nparams, lr, b1, b2, eps, c1, c2);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// ---------------------------------------------------------------------------------------------
// features: 16 numbers describing a CSR (rows = destinations for pull).  All from the device.
// ---------------------------------------------------------------------------------------------
// sums[0..]: rows, edges, sum d^2, max d, rows d=0, d in 1..7, 8..15, 16..31, >=32,
//            out-dangling, sum |src - row| (as double), max out, sum out^2
__global__ void k_feature_sums(const int32_t *rowptr, const int32_t *colidx, int64_t R, const int32_t *rowid,
                               const int32_t *out_rowptr, int32_t V, double *sums) {
    __shared__ double red[32];
    double s_d2 = 0, s_z = 0, s_b1 = 0, s_b2 = 0, s_b3 = 0, s_b4 = 0, s_loc = 0, s_dang = 0, s_o2 = 0;
    double mx = 0, mxo = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = rowptr[r + 1] - rowptr[r];
        s_d2 += (double)d * d;
        mx = fmax(mx, (double)d);
        s_z += d == 0;
        s_b1 += d >= 1 && d <= 7;
        s_b2 += d >= 8 && d <= 15;
        s_b3 += d >= 16 && d <= 31;
        s_b4 += d >= 32;
        const int64_t me = rowid ? rowid[r] : r;
        if (d > 0) s_loc += fabs((double)colidx[rowptr[r]] - (double)me);
    }
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; out_rowptr && v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t od = out_rowptr[v + 1] - out_rowptr[v];
        s_dang += od == 0;
        s_o2 += (double)od * od;
        mxo = fmax(mxo, (double)od);
    }
    double vals[11] = {s_d2, s_z, s_b1, s_b2, s_b3, s_b4, s_loc, s_dang, s_o2, mx, mxo};
    for (int i = 0; i < 9; ++i) {
        const double t = block_sum<double>(vals[i], red);
        if (threadIdx.x == 0) atomicAdd(sums + i, t);
    }
    for (int i = 9; i < 11; ++i) {
        double t = vals[i];
        for (int d = 16; d > 0; d >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, d));
        if ((threadIdx.x & 31) == 0) {
            unsigned long long *p = reinterpret_cast<unsigned long long *>(sums + i);
            atomicMax(p, (unsigned long long)t);  // stored as integer counts
        }
    }
}

static int features_impl(const int32_t *rowptr, const int32_t *colidx, int64_t R, int64_t E, const int32_t *rowid,
                         int32_t V, const int32_t *out_rowptr, int64_t l2_bytes, float *f, cudaStream_t s) {
    DevBuf sums;
    TC_TRY(sums.alloc(16 * 8));
    TC_CUDA(cudaMemsetAsync(sums.p, 0, 16 * 8, s));
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    k_feature_sums<<<caps.sms * 4, 256, 0, s>>>(rowptr, colidx, R, rowid, out_rowptr, V, sums.as<double>());
    TC_LAUNCH_CHECK();
    double h[16];
    TC_CUDA(cudaMemcpyAsync(h, sums.p, 16 * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    const double mxd = (double)reinterpret_cast<unsigned long long &>(h[9]);
    const double mxo = (double)reinterpret_cast<unsigned long long &>(h[10]);
    const double Rr = R > 0 ? (double)R : 1.0, Ee = E > 0 ? (double)E : 1.0, Vv = V > 0 ? (double)V : 1.0;
    const double mean = (double)E / Rr;
    const double var = h[0] / Rr - mean * mean;
    const double omean = (double)E / Vv;
    const double ovar = h[8] / Vv - omean * omean;
    f[0] = (float)log2(Rr + 1);
    f[1] = (float)log2(Ee + 1);
    f[2] = (float)mean;
    f[3] = (float)(mean > 0 ? sqrt(var > 0 ? var : 0) / mean : 0);
    f[4] = (float)log2(1 + mxd / (mean > 0 ? mean : 1));
    f[5] = (float)(h[1] / Rr);
    f[6] = (float)(h[2] / Rr);
    f[7] = (float)(h[3] / Rr);
    f[8] = (float)(h[4] / Rr);
    f[9] = (float)(h[5] / Rr);
    f[10] = (float)(omean > 0 ? sqrt(ovar > 0 ? ovar : 0) / omean : 0);
    f[11] = (float)(h[7] / Vv);
    f[12] = (float)log2(1 + 4.0 * Vv / (double)l2_bytes);
    f[13] = (float)log2(1 + 4.0 * Ee / (double)l2_bytes);
    f[14] = (float)(h[6] / (Rr * Vv));
    f[15] = (float)log2(1 + mxo / (omean > 0 ? omean : 1));
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_heads, const int32_t *head_sizes, tc_mlp **out) {
    using namespace tc;
    if (!out || !head_sizes || n_in < 1 || n_hidden < 1 || n_heads < 1 || n_heads > 8)
        return fail(TC_ERR_INVALID_ARG, "tc_mlp_create: bad sizes");
    *out = nullptr;
    tc_mlp *m = new (std::nothrow) tc_mlp();
    if (!m) return fail(TC_ERR_OOM, "host allocation failed");
    m->nin = n_in;
    m->nhid = n_hidden;
    m->nheads = n_heads;
    m->nout = 0;
    for (int k = 0; k < n_heads; ++k) {
        if (head_sizes[k] < 1) {
            delete m;
            return fail(TC_ERR_INVALID_ARG, "tc_mlp_create: empty head");
        }
        m->head_sizes[k] = head_sizes[k];
        m->nout += head_sizes[k];
    }
    m->nparams = mlp_offsets(m).total;
    const size_t pb = (size_t)m->nparams * 4;
    int st = m->params.alloc(pb);
    if (st == TC_OK) st = m->grads.alloc(pb);
    if (st == TC_OK) st = m->adam_m.alloc(pb);
    if (st == TC_OK) st = m->adam_v.alloc(pb);
    if (st == TC_OK && cudaMemset(m->params.p, 0, pb) != cudaSuccess) st = fail(TC_ERR_CUDA, "memset failed");
    if (st == TC_OK && cudaMemset(m->grads.p, 0, pb) != cudaSuccess) st = fail(TC_ERR_CUDA, "memset failed");
    if (st == TC_OK && cudaMemset(m->adam_m.p, 0, pb) != cudaSuccess) st = fail(TC_ERR_CUDA, "memset failed");
    if (st == TC_OK && cudaMemset(m->adam_v.p, 0, pb) != cudaSuccess) st = fail(TC_ERR_CUDA, "memset failed");
    if (st != TC_OK) {
        delete m;
        return st;
    }
    *out = m;
    return TC_OK;
}

extern "C" void tc_mlp_free(tc_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    delete m;
}

extern "C" int64_t tc_mlp_num_params(const tc_mlp *m) { return m ? m->nparams : -1; }

extern "C" int tc_mlp_set_params(tc_mlp *m, const float *params) {
    using namespace tc;
    if (!m || !params) return fail(TC_ERR_INVALID_ARG, "tc_mlp_set_params: null argument");
    TC_CUDA(cudaMemcpy(m->params.p, params, (size_t)m->nparams * 4, cudaMemcpyHostToDevice));
    TC_CUDA(cudaMemset(m->adam_m.p, 0, (size_t)m->nparams * 4));
    TC_CUDA(cudaMemset(m->adam_v.p, 0, (size_t)m->nparams * 4));
    m->step = 0;
    return TC_OK;
}

extern "C" int tc_mlp_get_params(const tc_mlp *m, float *params, float *grads) {
    using namespace tc;
    if (!m) return fail(TC_ERR_INVALID_ARG, "tc_mlp_get_params: null handle");
    if (params) TC_CUDA(cudaMemcpy(params, m->params.p, (size_t)m->nparams * 4, cudaMemcpyDeviceToHost));
    if (grads) TC_CUDA(cudaMemcpy(grads, m->grads.p, (size_t)m->nparams * 4, cudaMemcpyDeviceToHost));
    return TC_OK;
}

extern "C" int tc_mlp_forward(tc_mlp *m, const float *X, int32_t N, float *Z, int mem, void *stream) {
    using namespace tc;
    if (!m || !X || !Z || N < 1) return fail(TC_ERR_INVALID_ARG, "tc_mlp_forward: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    MlpWork w;
    TC_TRY(mlp_work(m, N, &w));
    TC_TRY(copy_to_dev(w.X, X, (size_t)N * m->nin * 4, mem, s));
    TC_TRY(mlp_forward_dev(m, w, N, s));
    TC_CUDA(cudaMemcpyAsync(Z, w.Z, (size_t)N * m->nout * 4,
                            mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

extern "C" int tc_mlp_loss_grad(tc_mlp *m, const float *X, const int32_t *Y, int32_t N, int mem, double *loss,
                                void *stream) {
    using namespace tc;
    if (!m || !X || !Y || N < 1) return fail(TC_ERR_INVALID_ARG, "tc_mlp_loss_grad: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    MlpWork w;
    TC_TRY(mlp_work(m, N, &w));
    TC_TRY(copy_to_dev(w.X, X, (size_t)N * m->nin * 4, mem, s));
    TC_TRY(copy_to_dev(w.Y, Y, (size_t)N * m->nheads * 4, mem, s));
    TC_TRY(check_labels(m, w.Y, N, s));
    TC_TRY(mlp_loss_grad_dev(m, w, N, true, s));
    double l = 0;
    TC_CUDA(cudaMemcpyAsync(&l, w.loss_sum, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (loss) *loss = l / N;
    return TC_OK;
}

extern "C" int tc_mlp_adam_step(tc_mlp *m, float lr, float beta1, float beta2, float eps, void *stream) {
    using namespace tc;
    if (!m) return fail(TC_ERR_INVALID_ARG, "tc_mlp_adam_step: null handle");
    TC_TRY(adam_dev(m, lr, beta1, beta2, eps, (cudaStream_t)stream));
    return TC_OK;
}

extern "C" int tc_mlp_train(tc_mlp *m, const float *X, const int32_t *Y, int32_t N, int32_t epochs, int32_t batch,
                            float lr, int mem, double *final_loss, void *stream) {
    using namespace tc;
    if (!m || !X || !Y || N < 1 || epochs < 0 || batch < 1) return fail(TC_ERR_INVALID_ARG, "tc_mlp_train: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf Xall, Yall;
    TC_TRY(Xall.alloc((size_t)N * m->nin * 4));
    TC_TRY(Yall.alloc((size_t)N * m->nheads * 4));
    TC_TRY(copy_to_dev(Xall.p, X, (size_t)N * m->nin * 4, mem, s));
    TC_TRY(copy_to_dev(Yall.p, Y, (size_t)N * m->nheads * 4, mem, s));
    TC_TRY(check_labels(m, Yall.as<int32_t>(), N, s));
    MlpWork w;
    const int32_t B = batch < N ? batch : N;
    TC_TRY(mlp_work(m, B, &w));
    for (int32_t ep = 0; ep < epochs; ++ep) {
        for (int32_t b0 = 0; b0 < N; b0 += B) {  // the caller orders the samples (shuffled per epoch upstream)
            const int32_t nb = (N - b0) < B ? (N - b0) : B;
            TC_CUDA(cudaMemcpyAsync(w.X, Xall.as<float>() + (int64_t)b0 * m->nin, (size_t)nb * m->nin * 4,
                                    cudaMemcpyDeviceToDevice, s));
            TC_CUDA(cudaMemcpyAsync(w.Y, Yall.as<int32_t>() + (int64_t)b0 * m->nheads, (size_t)nb * m->nheads * 4,
                                    cudaMemcpyDeviceToDevice, s));
            TC_TRY(mlp_loss_grad_dev(m, w, nb, true, s));
            TC_TRY(adam_dev(m, lr, 0.9f, 0.999f, 1e-8f, s));
        }
    }
    // final loss over the whole set
    MlpWork wf;
    TC_TRY(mlp_work(m, N, &wf));
    TC_CUDA(cudaMemcpyAsync(wf.X, Xall.p, (size_t)N * m->nin * 4, cudaMemcpyDeviceToDevice, s));
    TC_CUDA(cudaMemcpyAsync(wf.Y, Yall.p, (size_t)N * m->nheads * 4, cudaMemcpyDeviceToDevice, s));
    TC_TRY(mlp_loss_grad_dev(m, wf, N, false, s));
    double l = 0;
    TC_CUDA(cudaMemcpyAsync(&l, wf.loss_sum, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (final_loss) *final_loss = l / N;
    return TC_OK;
}

extern "C" int tc_graph_features(const tc_graph *g, float *features) {
    using namespace tc;
    if (!g || !features) return fail(TC_ERR_INVALID_ARG, "tc_graph_features: null argument");
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    return features_impl(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), g->V, g->E, nullptr, g->V,
                         g->out_rowptr.as<int32_t>(), caps.l2_bytes, features, nullptr);
}

extern "C" int tc_part_features(const tc_part *p, float *features) {
    using namespace tc;
    if (!p || !features) return fail(TC_ERR_INVALID_ARG, "tc_part_features: null argument");
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    const tc_graph *g = p->g;
    float gf[16];
    TC_TRY(features_impl(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), g->V, g->E, nullptr, g->V,
                         g->out_rowptr.as<int32_t>(), caps.l2_bytes, gf, nullptr));
    for (int32_t b = 0; b < p->B; ++b) {
        const int64_t r0 = p->h_blk_rows[b], r1 = p->h_blk_rows[b + 1];
        const int64_t e0 = p->h_blk_edges[b], e1 = p->h_blk_edges[b + 1];
        float *f = features + (int64_t)b * 16;
        // rows of one block (row ids through id_map); the out-degree features are the graph's
        TC_TRY(features_impl(p->rowptr.as<int32_t>() + r0, p->colidx.as<int32_t>(), r1 - r0, e1 - e0,
                             p->id_map.as<int32_t>() + r0, g->V, nullptr, caps.l2_bytes, f, nullptr));
        f[10] = gf[10];
        f[11] = gf[11];
        f[15] = gf[15];
        f[12] = (float)log2(1 + 4.0 * (double)p->W / (double)caps.l2_bytes);  // the block's vertex values
    }
    return TC_OK;
}
