// lcq_pred.cu -- hierarchical-grid prediction of quantization bins, the
// project's extension (the paper stores bins as they are and leaves
// decorrelation to LC's later stages; it has no counterpart for this part).
//
// Definition (the same one the oracle implements independently):
//   * N x N x N int32 bins, index (i*N + j)*N + k.  Anchors: all coordinates
//     multiples of 8, kept as they are.  A point of stride s in {4, 2, 1}
//     (level 1, 2, 3) has coordinates that are multiples of s, not all
//     multiples of 2s; its class is the bit set of its odd axes (coordinate /
//     s odd; bit 0 = i, bit 1 = j, bit 2 = k).
//   * Coarse positions on an axis are clamped to [0, last], last = the largest
//     multiple of 2s not above N-1.
//   * Interpolation: (sum of the 2^c corner bins p +/- s along the odd axes
//     + 2^(c-1)) >> c, in 64-bit.
//   * Network (one int8 weight set per level and class): inputs
//     x_t = clamp((bin of coarse stencil point t - base) >> s_in, -128, 127)
//     over the 3x3x3 coarse points f + 2s (di, dj, dk) around the floor-aligned
//     coarse point f; h_u = clamp((W1 x + b1 + 2^(s1-1)) >> s1, 0, 127);
//     o = (W2 h + b2 + 2^(s2-1)) >> s2; pred = base + o.  Dot products use
//     __dp4a (4 int8 products into an int32 accumulator, exact).
//   * Residual = bin - pred modulo 2^32; reconstruction adds it back level by
//     level.
//   * Training: shadow parameters in float32 (integer units), forward pass =
//     the exact integer network on rint/clamped parameters (every sum is an
//     integer below 2^24, so float32 holds it exactly), loss = mean squared
//     residual, straight-through gradients; per-CTA partial gradients are
//     summed in a fixed order (deterministic), then Adam.
#include <cmath>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/lcq.h"

namespace lcq {
namespace pred {

constexpr int kNin = 27, kNhid = 16, kNets = 21;
constexpr int kHistHalf = 1 << 20;   // histogram covers [-2^20, 2^20)
constexpr int kSmemHistHalf = 4096;  // per-block histogram of the centre range
constexpr int kTrainBlock = 256;
constexpr int kNparam = kNhid * kNin + kNhid + kNhid + 1;  // 465

static_assert(sizeof(lcq_pred_params) == 3 * 7 * 16 * 28 + 3 * 7 * 16 * 4 + 3 * 7 * 16 + 3 * 7 * 4 + 6 * 4,
              "lcq_pred_params layout");

struct Point {
    int level;  // 0 anchor, 1..3
    int s;      // stride
    int cls;    // 1..7
};

__device__ __forceinline__ Point classify(int i, int j, int k) {
    const int m = (i | j | k) & 7;
    Point p;
    if (m == 0) {
        p.level = 0; p.s = 8; p.cls = 0;
        return p;
    }
    p.s = m & (-m);
    p.level = p.s == 4 ? 1 : (p.s == 2 ? 2 : 3);
    p.cls = ((i & p.s) ? 1 : 0) | ((j & p.s) ? 2 : 0) | ((k & p.s) ? 4 : 0);
    return p;
}

__device__ __forceinline__ int clampc(int v, int last) { return v < 0 ? 0 : (v > last ? last : v); }

__device__ __forceinline__ int32_t at(const int32_t* b, int N, int i, int j, int k) {
    return b[((size_t)i * N + j) * N + k];
}

// Element offset, relative to point (i, j, k), of a coarse position along
// each axis: ((ci - i) N + (cj - j)) N + (ck - k), split per axis.  The
// positions lie within 2 s2 <= 16 of the point, so each term fits in int32
// for N <= 2048.
__device__ __forceinline__ int axis_off(int c, int x, int stride) { return (c - x) * stride; }

// Interpolation base of point (i, j, k) (not an anchor); p = &b[i][j][k].
__device__ __forceinline__ int32_t interp(const int32_t* p, int N, int i, int j, int k, const Point& pt) {
    const int s = pt.s, last = ((N - 1) / (2 * s)) * (2 * s), NN = N * N;
    const int i0 = (pt.cls & 1) ? axis_off(clampc(i - s, last), i, NN) : 0;
    const int i1 = (pt.cls & 1) ? axis_off(clampc(i + s, last), i, NN) : 0;
    const int j0 = (pt.cls & 2) ? axis_off(clampc(j - s, last), j, N) : 0;
    const int j1 = (pt.cls & 2) ? axis_off(clampc(j + s, last), j, N) : 0;
    const int k0 = (pt.cls & 4) ? clampc(k - s, last) - k : 0;
    const int k1 = (pt.cls & 4) ? clampc(k + s, last) - k : 0;
    const int c = __popc(pt.cls);
    long long acc = 0;
    // enumerate the 2^c distinct corners: along an even axis both ends coincide
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if ((q & ~pt.cls) != 0) continue;
        acc += p[((q & 1) ? i1 : i0) + ((q & 2) ? j1 : j0) + ((q & 4) ? k1 : k0)];
    }
    return (int32_t)((acc + (1ll << (c - 1))) >> c);
}

// The 27 stencil inputs packed 4 per int32 (byte 3 of word 6 is 0);
// p = &b[i][j][k].
__device__ __forceinline__ void stencil(const int32_t* p, int N, int i, int j, int k, const Point& pt,
                                        int32_t base, int s_in, int32_t xw[7]) {
    const int s2 = 2 * pt.s, last = ((N - 1) / s2) * s2, NN = N * N;
    const int fi = (i / s2) * s2, fj = (j / s2) * s2, fk = (k / s2) * s2;
    int oi[3], oj[3], ok[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        oi[d] = axis_off(clampc(fi + s2 * (d - 1), last), i, NN);
        oj[d] = axis_off(clampc(fj + s2 * (d - 1), last), j, N);
        ok[d] = clampc(fk + s2 * (d - 1), last) - k;
    }
#pragma unroll
    for (int w = 0; w < 7; w++) xw[w] = 0;
#pragma unroll
    for (int t = 0; t < kNin; t++) {
        const int32_t c = p[oi[t / 9] + oj[(t / 3) % 3] + ok[t % 3]];
        int32_t d = (c - base) >> s_in;  // |c - base| < 2^31: both bins lie in (-2^30, 2^30)
        d = d < -128 ? -128 : (d > 127 ? 127 : d);
        xw[t >> 2] |= (int32_t)((uint32_t)(d & 0xFF) << (8 * (t & 3)));
    }
}

// Parameters in shared memory, W1 rows as 7 packed int32 words and a zero
// eighth, so that a row is two 16-byte loads.
struct SmemParams {
    int4 w1[kNets][kNhid][2];
    int32_t b1[kNets][kNhid];
    int32_t w2[kNets][4];
    int32_t b2[kNets];
    int32_t s_in[3];
    int32_t s1, s2;
};

__device__ __forceinline__ void load_params(SmemParams& sp, const lcq_pred_params* gp) {
    const int32_t* w1 = reinterpret_cast<const int32_t*>(gp->w1);
    const int32_t* w2 = reinterpret_cast<const int32_t*>(gp->w2);
    int32_t* sw1 = reinterpret_cast<int32_t*>(&sp.w1[0][0][0]);
    for (int x = threadIdx.x; x < kNets * kNhid * 8; x += blockDim.x) sw1[x] = (x & 7) < 7 ? w1[(x >> 3) * 7 + (x & 7)] : 0;
    for (int x = threadIdx.x; x < kNets * kNhid; x += blockDim.x) (&sp.b1[0][0])[x] = (&gp->b1[0][0][0])[x];
    for (int x = threadIdx.x; x < kNets * 4; x += blockDim.x) (&sp.w2[0][0])[x] = w2[x];
    for (int x = threadIdx.x; x < kNets; x += blockDim.x) sp.b2[x] = (&gp->b2[0][0])[x];
    if (threadIdx.x < 3) sp.s_in[threadIdx.x] = gp->s_in[threadIdx.x];
    if (threadIdx.x == 0) { sp.s1 = gp->s1; sp.s2 = gp->s2; }
}

__device__ __forceinline__ int32_t network(const SmemParams& sp, int net, const int32_t xw[7]) {
    int32_t hw[4] = {0, 0, 0, 0};
#pragma unroll
    for (int u = 0; u < kNhid; u++) {
        int32_t z = sp.b1[net][u];
        const int4 a = sp.w1[net][u][0], c = sp.w1[net][u][1];
        z = __dp4a(xw[0], a.x, z);
        z = __dp4a(xw[1], a.y, z);
        z = __dp4a(xw[2], a.z, z);
        z = __dp4a(xw[3], a.w, z);
        z = __dp4a(xw[4], c.x, z);
        z = __dp4a(xw[5], c.y, z);
        z = __dp4a(xw[6], c.z, z);
        int32_t h = (z + (1 << (sp.s1 - 1))) >> sp.s1;
        h = h < 0 ? 0 : (h > 127 ? 127 : h);
        hw[u >> 2] |= h << (8 * (u & 3));
    }
    int32_t o = sp.b2[net];
#pragma unroll
    for (int w = 0; w < 4; w++) o = __dp4a(hw[w], sp.w2[net][w], o);
    return (o + (1 << (sp.s2 - 1))) >> sp.s2;
}

__device__ __forceinline__ int32_t predict_point(const int32_t* b, int N, int i, int j, int k, const Point& pt,
                                                 const SmemParams* sp) {
    const int32_t* p = b + (((size_t)i * N + j) * N + k);
    int32_t base = interp(p, N, i, j, k, pt);
    if (sp) {
        int32_t xw[7];
        stencil(p, N, i, j, k, pt, base, sp->s_in[pt.level - 1], xw);
        base = (int32_t)((uint32_t)base + (uint32_t)network(*sp, (pt.level - 1) * 7 + (pt.cls - 1), xw));
    }
    return base;
}

// ---------------------------------------------------------------- kernels --

template <bool NET>
__global__ void __launch_bounds__(256) k_residuals(const int32_t* __restrict__ bins, int N,
                                                   const lcq_pred_params* params, int32_t* __restrict__ res) {
    __shared__ SmemParams sp;
    if (NET) {
        load_params(sp, params);
        __syncthreads();
    }
    const int i = blockIdx.z, j = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const size_t e = ((size_t)i * N + j) * N + k;
        const Point pt = classify(i, j, k);
        if (pt.level == 0) {
            res[e] = bins[e];
        } else {
            const int32_t pr = predict_point(bins, N, i, j, k, pt, NET ? &sp : nullptr);
            res[e] = (int32_t)((uint32_t)bins[e] - (uint32_t)pr);
        }
    }
}

// Reconstruct the points of one level (anchors when s == 8) on the lattice of
// multiples of s.
template <bool NET>
__global__ void __launch_bounds__(256) k_reconstruct(const int32_t* __restrict__ res, int N, int s,
                                                     const lcq_pred_params* params, int32_t* bins) {
    __shared__ SmemParams sp;
    if (NET) {
        load_params(sp, params);
        __syncthreads();
    }
    const int i = blockIdx.z * s, j = blockIdx.y * s;
    for (int kk = blockIdx.x * blockDim.x + threadIdx.x; kk * s < N; kk += gridDim.x * blockDim.x) {
        const int k = kk * s;
        const Point pt = classify(i, j, k);
        if (pt.s != s) continue;  // belongs to another level
        const size_t e = ((size_t)i * N + j) * N + k;
        if (pt.level == 0) {
            bins[e] = res[e];
        } else {
            const int32_t pr = predict_point(bins, N, i, j, k, pt, NET ? &sp : nullptr);
            bins[e] = (int32_t)((uint32_t)pr + (uint32_t)res[e]);
        }
    }
}

// Histograms of residuals over [-2^20, 2^20): hist[0] anchors, hist[1]
// predicted points; outliers (mask bit set) are skipped; values outside the
// range are counted in over[0] / over[1].
__global__ void __launch_bounds__(256) k_histogram(const int32_t* __restrict__ res, int N,
                                                   const uint32_t* __restrict__ mask, uint32_t* hist,
                                                   unsigned long long* over) {
    __shared__ uint32_t sh[2 * kSmemHistHalf];
    for (int x = threadIdx.x; x < 2 * kSmemHistHalf; x += blockDim.x) sh[x] = 0;
    __syncthreads();
    const int i = blockIdx.z, j = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const size_t e = ((size_t)i * N + j) * N + k;
        if (mask && ((mask[e >> 5] >> (e & 31)) & 1u)) continue;
        const bool anchor = ((i | j | k) & 7) == 0;
        const int32_t v = res[e];
        uint32_t* h = hist + (anchor ? 0 : 2 * kHistHalf);
        if (!anchor && v >= -kSmemHistHalf / 2 && v < kSmemHistHalf / 2) {
            atomicAdd(&sh[v + kSmemHistHalf / 2], 1u);
        } else if (v >= -kHistHalf && v < kHistHalf) {
            atomicAdd(&h[v + kHistHalf], 1u);
        } else {
            atomicAdd(&over[anchor ? 0 : 1], 1ull);
        }
    }
    __syncthreads();
    uint32_t* h = hist + 2 * kHistHalf;
    for (int x = threadIdx.x; x < kSmemHistHalf; x += blockDim.x)
        if (sh[x]) atomicAdd(&h[x - kSmemHistHalf / 2 + kHistHalf], sh[x]);
}

// ---------------------------------------------------------------- training --

struct TrainItem {
    uint32_t net;    // (level-1)*7 + (class-1)
    uint32_t start;  // first sample
    uint32_t count;  // <= kTrainBlock
    uint32_t pad;
};

struct TParams {
    const int32_t* bins;        // fields back to back, N^3 each
    int N;
    const uint64_t* samples;    // (field << 32) | flat point index, grouped by network
    const TrainItem* items;
    const float* shadow;        // [kNets][kNparam]: w1[16][27], b1[16], w2[16], b2
    const float* inv_count;     // [kNets]: 1 / samples of that network
    int32_t s_in[3];
    int32_t s1, s2;
    float* partial;             // [items][kNparam + 1]; last = loss sum
};

__global__ void __launch_bounds__(kTrainBlock) k_train_partial(TParams p) {
    extern __shared__ float tsm[];
    float* s_go = tsm;                                   // [256]
    float* s_h = s_go + kTrainBlock;                     // [256][16]
    float* s_gz = s_h + kTrainBlock * kNhid;             // [256][16]
    float* s_x = s_gz + kTrainBlock * kNhid;             // [256][27]
    float* s_r2 = s_x + kTrainBlock * kNin;              // [256]
    float* s_w = s_r2 + kTrainBlock;                     // fake-quantised params [kNparam]
    float* s_m = s_w + kNparam;                          // straight-through masks [kNparam]
    const TrainItem it = p.items[blockIdx.x];
    const float* sh = p.shadow + (size_t)it.net * kNparam;
    const float lim[4] = {127.0f, 4194304.0f, 127.0f, 4194304.0f};
    for (int q = threadIdx.x; q < kNparam; q += blockDim.x) {
        const int part = q < kNhid * kNin ? 0 : (q < kNhid * kNin + kNhid ? 1 : (q < kNparam - 1 ? 2 : 3));
        const float lo = part == 0 || part == 2 ? -128.0f : -lim[part];
        const float r = rintf(sh[q]);
        s_m[q] = (r >= lo && r <= lim[part]) ? 1.0f : 0.0f;
        s_w[q] = fminf(fmaxf(r, lo), lim[part]);
    }
    __syncthreads();
    const int level = (int)(it.net / 7) + 1, cls = (int)(it.net % 7) + 1;
    const float* W1 = s_w;
    const float* B1 = s_w + kNhid * kNin;
    const float* W2 = B1 + kNhid;
    const float B2 = W2[kNhid];
    const float sc1 = ldexpf(1.0f, -p.s1), sc2 = ldexpf(1.0f, -p.s2);
    const int t = threadIdx.x;
    if (t < (int)it.count) {
        const uint64_t smp = p.samples[it.start + t];
        const uint32_t f = (uint32_t)(smp >> 32), e = (uint32_t)smp;
        const int N = p.N;
        const int i = (int)(e / ((uint32_t)N * N)), j = (int)((e / N) % N), k = (int)(e % N);
        const int32_t* b = p.bins + (size_t)f * N * N * N;
        Point pt = classify(i, j, k);
        (void)level; (void)cls;
        const int32_t* pp = b + (size_t)e;
        const int32_t base = interp(pp, N, i, j, k, pt);
        int32_t xw[7];
        stencil(pp, N, i, j, k, pt, base, p.s_in[pt.level - 1], xw);
        float x[kNin];
#pragma unroll
        for (int q = 0; q < kNin; q++) x[q] = (float)(int8_t)((xw[q >> 2] >> (8 * (q & 3))) & 0xFF);
        float h[kNhid], on[kNhid];
#pragma unroll
        for (int u = 0; u < kNhid; u++) {
            float z = B1[u];
#pragma unroll
            for (int q = 0; q < kNin; q++) z = __fadd_rn(z, __fmul_rn(W1[u * kNin + q], x[q]));  // exact integers
            const float hu = floorf(__fmul_rn(__fadd_rn(z, ldexpf(1.0f, p.s1 - 1)), sc1));
            on[u] = (hu > 0.0f && hu < 127.0f) ? 1.0f : 0.0f;
            h[u] = fminf(fmaxf(hu, 0.0f), 127.0f);
        }
        float acc = B2;
#pragma unroll
        for (int u = 0; u < kNhid; u++) acc = __fadd_rn(acc, __fmul_rn(W2[u], h[u]));
        const float o = floorf(__fmul_rn(__fadd_rn(acc, ldexpf(1.0f, p.s2 - 1)), sc2));
        const long long rr = (long long)b[e] - ((long long)base + (long long)o);
        const float r = (float)rr;
        const float go = -2.0f * r * p.inv_count[it.net];
        s_go[t] = go;
        s_r2[t] = r * r;
#pragma unroll
        for (int u = 0; u < kNhid; u++) {
            s_h[t * kNhid + u] = h[u];
            s_gz[t * kNhid + u] = go * W2[u] * sc2 * on[u] * sc1;
        }
#pragma unroll
        for (int q = 0; q < kNin; q++) s_x[t * kNin + q] = x[q];
    }
    __syncthreads();
    // per-parameter sums over this item's samples, in sample order
    float* out = p.partial + (size_t)blockIdx.x * (kNparam + 1);
    for (int q = threadIdx.x; q <= kNparam; q += blockDim.x) {
        float acc = 0.0f;
        if (q < kNhid * kNin) {
            const int u = q / kNin, c = q % kNin;
            for (uint32_t s = 0; s < it.count; s++) acc += s_gz[s * kNhid + u] * s_x[s * kNin + c];
        } else if (q < kNhid * kNin + kNhid) {
            const int u = q - kNhid * kNin;
            for (uint32_t s = 0; s < it.count; s++) acc += s_gz[s * kNhid + u];
        } else if (q < kNparam - 1) {
            const int u = q - kNhid * kNin - kNhid;
            for (uint32_t s = 0; s < it.count; s++) acc += s_go[s] * s_h[s * kNhid + u];
            acc *= sc2;
        } else if (q == kNparam - 1) {
            for (uint32_t s = 0; s < it.count; s++) acc += s_go[s];
            acc *= sc2;
        } else {
            for (uint32_t s = 0; s < it.count; s++) acc += s_r2[s];
        }
        out[q] = q < kNparam ? acc * s_m[q] : acc;
    }
}

// grad[net][q] = sum over the items of net (in item order) of partial[item][q]
__global__ void k_train_reduce(const float* partial, const uint32_t* item_begin, float* grad, float* loss) {
    const int net = blockIdx.x;
    for (int q = threadIdx.x; q <= kNparam; q += blockDim.x) {
        float acc = 0.0f;
        for (uint32_t it = item_begin[net]; it < item_begin[net + 1]; it++) acc += partial[(size_t)it * (kNparam + 1) + q];
        if (q < kNparam) grad[(size_t)net * kNparam + q] = acc;
        else loss[net] = acc;
    }
}

// Adam (Kingma & Ba, 2015) on the shadow parameters.
__global__ void k_adam(float* w, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// Shadow parameters -> packed int8 network (rint, clamp).
__global__ void k_freeze(const float* shadow, lcq_pred_params* out) {
    const int net = blockIdx.x, lv = net / 7, cl = net % 7;
    const float* sh = shadow + (size_t)net * kNparam;
    for (int q = threadIdx.x; q < kNhid * 28; q += blockDim.x) {
        const int u = q / 28, c = q % 28;
        out->w1[lv][cl][u][c] = c < kNin ? (int8_t)fminf(fmaxf(rintf(sh[u * kNin + c]), -128.0f), 127.0f) : 0;
    }
    for (int u = threadIdx.x; u < kNhid; u += blockDim.x) {
        out->b1[lv][cl][u] = (int32_t)fminf(fmaxf(rintf(sh[kNhid * kNin + u]), -4194304.0f), 4194304.0f);
        out->w2[lv][cl][u] = (int8_t)fminf(fmaxf(rintf(sh[kNhid * kNin + kNhid + u]), -128.0f), 127.0f);
    }
    if (threadIdx.x == 0) out->b2[lv][cl] = (int32_t)fminf(fmaxf(rintf(sh[kNparam - 1]), -4194304.0f), 4194304.0f);
}

static bool n_ok(int N) { return N >= 1 && N <= 2048; }

}  // namespace pred
}  // namespace lcq

using namespace lcq::pred;

extern "C" {

lcq_status lcq_pred_residuals(const int32_t* d_bins, uint32_t N, const lcq_pred_params* d_params, int32_t* d_res,
                              cudaStream_t stream) {
    if (!n_ok((int)N) || !d_bins || !d_res) return LCQ_ERR_ARG;
    const dim3 grid((N + 255) / 256, N, N);
    if (d_params) k_residuals<true><<<grid, 256, 0, stream>>>(d_bins, (int)N, d_params, d_res);
    else k_residuals<false><<<grid, 256, 0, stream>>>(d_bins, (int)N, nullptr, d_res);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_pred_reconstruct(const int32_t* d_res, uint32_t N, const lcq_pred_params* d_params, int32_t* d_bins,
                                cudaStream_t stream) {
    if (!n_ok((int)N) || !d_bins || !d_res) return LCQ_ERR_ARG;
    for (int s : {8, 4, 2, 1}) {
        const unsigned m = (N + s - 1) / s;
        const dim3 grid((m + 255) / 256, m, m);
        if (d_params) k_reconstruct<true><<<grid, 256, 0, stream>>>(d_res, (int)N, s, d_params, d_bins);
        else k_reconstruct<false><<<grid, 256, 0, stream>>>(d_res, (int)N, s, nullptr, d_bins);
        if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    }
    return LCQ_OK;
}

size_t lcq_pred_histogram_words(void) { return 4ull * kHistHalf; }

lcq_status lcq_pred_histogram(const int32_t* d_res, uint32_t N, const uint32_t* d_mask, uint32_t* d_hist,
                              unsigned long long* d_over, cudaStream_t stream) {
    if (!n_ok((int)N) || !d_res || !d_hist || !d_over) return LCQ_ERR_ARG;
    if (cudaMemsetAsync(d_hist, 0, 4ull * kHistHalf * sizeof(uint32_t), stream) != cudaSuccess ||
        cudaMemsetAsync(d_over, 0, 2 * sizeof(unsigned long long), stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    const dim3 grid((N + 255) / 256, N, N);
    k_histogram<<<grid, 256, 0, stream>>>(d_res, (int)N, d_mask, d_hist, d_over);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_train_gradients(const int32_t* d_bins, uint32_t N, const uint64_t* d_samples, const void* d_items,
                               uint32_t num_items, const uint32_t* d_item_begin, const float* d_shadow,
                               const float* d_inv_count, const int32_t* h_s_in, int32_t s1, int32_t s2,
                               float* d_partial, float* d_grad, float* d_loss, cudaStream_t stream) {
    if (!n_ok((int)N) || !d_bins || !d_samples || !d_items || !d_item_begin || !d_shadow || !d_inv_count ||
        !h_s_in || !d_partial || !d_grad || !d_loss || s1 < 1 || s1 > 24 || s2 < 1 || s2 > 24)
        return LCQ_ERR_ARG;
    TParams p;
    p.bins = d_bins;
    p.N = (int)N;
    p.samples = d_samples;
    p.items = reinterpret_cast<const TrainItem*>(d_items);
    p.shadow = d_shadow;
    p.inv_count = d_inv_count;
    for (int l = 0; l < 3; l++) {
        if (h_s_in[l] < 0 || h_s_in[l] > 30) return LCQ_ERR_ARG;
        p.s_in[l] = h_s_in[l];
    }
    p.s1 = s1;
    p.s2 = s2;
    p.partial = d_partial;
    const size_t smem = sizeof(float) * ((size_t)kTrainBlock * (2 + 2 * kNhid + kNin) + 2 * kNparam);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_train_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (num_items) k_train_partial<<<num_items, kTrainBlock, smem, stream>>>(p);
    if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    k_train_reduce<<<kNets, 256, 0, stream>>>(d_partial, d_item_begin, d_grad, d_loss);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_train_adam(float* d_shadow, float* d_m, float* d_v, const float* d_grad, float lr, float beta1,
                          float beta2, float eps, uint32_t step, cudaStream_t stream) {
    if (!d_shadow || !d_m || !d_v || !d_grad || step == 0) return LCQ_ERR_ARG;
    const int n = kNets * kNparam;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, stream>>>(d_shadow, d_m, d_v, d_grad, n, lr, beta1, beta2, eps, c1, c2);
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_pred_freeze(const float* d_shadow, const int32_t* h_s_in, int32_t s1, int32_t s2,
                           lcq_pred_params* d_params, cudaStream_t stream) {
    if (!d_shadow || !d_params || !h_s_in) return LCQ_ERR_ARG;
    int32_t tail[6] = {h_s_in[0], h_s_in[1], h_s_in[2], s1, s2, 0};
    k_freeze<<<kNets, 128, 0, stream>>>(d_shadow, d_params);
    if (cudaPeekAtLastError() != cudaSuccess) return LCQ_ERR_CUDA;
    // shifts: a small host-to-device copy from a stack buffer (synchronous w.r.t. the host buffer)
    if (cudaMemcpyAsync(&d_params->s_in[0], tail, sizeof(tail), cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return LCQ_ERR_CUDA;
    return cudaStreamSynchronize(stream) == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

uint32_t lcq_train_param_count(void) { return kNets * kNparam; }

}  // extern "C"
