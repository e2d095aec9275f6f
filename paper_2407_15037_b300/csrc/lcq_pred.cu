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
//     o = (W2 h + b2 + 2^(s2-1)) >> s2; pred = base + o.  Both products,
//     W1 x and W2 h, run on the tensor cores (binary16 operands, float32
//     accumulators, exact for these integers), the rest in integers.
//   * Residual = bin - pred modulo 2^32; reconstruction adds it back level by
//     level.
//   * Training: shadow parameters in float32 (integer units), forward pass =
//     the exact integer network on rint/clamped parameters (every sum is an
//     integer below 2^24, so float32 holds it exactly), loss = mean squared
//     residual, straight-through gradients; per-CTA partial gradients are
//     summed in a fixed order (deterministic), then Adam.
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstring>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/lcq.h"
#include "lcq_host.h"

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
    int sh;     // log2(2 s): coarse positions are the multiples of 1 << sh
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
    p.sh = __ffs(p.s);  // log2(s) + 1
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
    const int s = pt.s, last = ((N - 1) >> pt.sh) << pt.sh, NN = N * N;  // 2 s = 1 << sh
    // ends x - d and x + d with d = s on an odd axis and d = 0 on an even one
    // (an even coordinate is a multiple of 2s, so it is at most last)
    const int di = (pt.cls & 1) ? s : 0, dj = (pt.cls & 2) ? s : 0, dk = (pt.cls & 4) ? s : 0;
    const int i0 = axis_off(clampc(i - di, last), i, NN), i1 = axis_off(clampc(i + di, last), i, NN);
    const int j0 = axis_off(clampc(j - dj, last), j, N), j1 = axis_off(clampc(j + dj, last), j, N);
    const int k0 = clampc(k - dk, last) - k, k1 = clampc(k + dk, last) - k;
    // all 8 end combinations: along an even axis both ends are the point's own
    // coordinate, so each of the 2^c distinct corners (c odd axes) is added
    // 2^(3 - c) times and the mean (sum + 2^(c-1)) >> c is (acc + 4) >> 3.
    // Bins lie in (-2^30, 2^30), so the two k ends add up in int32.
    long long acc = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int32_t* r = p + ((q & 1) ? i1 : i0) + ((q & 2) ? j1 : j0);
        acc += (long long)(r[k0] + r[k1]);
    }
    return (int32_t)((acc + 4) >> 3);
}

// The 27 stencil inputs packed 4 per int32 (byte 3 of word 6 is 0);
// p = &b[i][j][k].
__device__ __forceinline__ void stencil(const int32_t* p, int N, int i, int j, int k, const Point& pt,
                                        int32_t base, int s_in, int32_t xw[7]) {
    const int s2 = 2 * pt.s, last = ((N - 1) >> pt.sh) << pt.sh, NN = N * N;  // s2 = 1 << sh
    const int fi = (i >> pt.sh) << pt.sh, fj = (j >> pt.sh) << pt.sh, fk = (k >> pt.sh) << pt.sh;
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

// Interpolation prediction of point (i, j, k) (not an anchor) from bins b.
__device__ __forceinline__ int32_t interp_point(const int32_t* b, int N, int i, int j, int k, const Point& pt) {
    return interp(b + (((size_t)i * N + j) * N + k), N, i, j, k, pt);
}

// ------------------------------------------------ network on tensor cores --
//
// A warp evaluates the network for 32 points of one (level, class) at once:
// hidden = W1 x as a [32 points x 32 inputs] x [32 inputs x 16 hidden]
// product on the tensor cores (mma.sync m16n8k16, binary16 operands, float32
// accumulators), then W2 h as a [32 points x 16 hidden] x [16 hidden x 8]
// product whose column 0 is W2; the shifts and clamps in integers.  The A
// operand holds 640 + x_t rather than x_t: for x_t in [-128, 127] that is an
// integer in [512, 767], where
// binary16 values are spaced 1/2 apart, so its bit pattern is just
// 0x6100 + 2 x_t (no conversion); the extra 640 sum_t W1[u][t] is taken off
// with the bias.  This is exact: the weights are integers in [-128, 127] and
// the inputs integers below 768, all exact in binary16; every product has
// magnitude below 2^17 and every partial sum of the 27 products is an
// integer below 27 * 128 * 767 < 2^22, exact in float32 whatever the order
// of the additions.  So each accumulator equals the integer dot product.

struct MmaParams {
    uint32_t bfrag[kNets][32][8];  // W1 as B fragments: [net][lane][n-tile * 4 + k-step * 2 + reg]
    uint32_t zk[kNets][kNhid];     // b1 + 2^(s1-1) - 640 sum_t W1[u][t] - bits(1.5 2^23), mod 2^32
    uint32_t w2frag[kNets][32][2]; // W2 as the B fragment of a 16 x 8 matrix whose column 0 is W2
    uint32_t b2k[kNets];           // b2 + 2^(s2-1) - 1024 sum_u W2[u] - bits(1.5 2^23), mod 2^32
    int32_t s_in[3];
    int32_t s1, s2;
};

constexpr int kArow = 20;  // words per point row of the A staging tile (16 used; 80 B rows: no bank conflicts)

// Two int8 weights as a binary16 pair (exact; .x = lo in the low half).
__device__ __forceinline__ uint32_t half_pair(int lo, int hi) {
    const __half2 v = __floats2half2_rn((float)lo, (float)hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Two inputs x in [-128, 127] as the binary16 pair (640 + lo, 640 + hi):
// bit patterns 0x6100 + 2 x; the low half never borrows from the high one.
__device__ __forceinline__ uint32_t input_pair(int lo, int hi) {
    return 0x61006100u + (uint32_t)(2 * lo) + ((uint32_t)hi << 17);
}

__device__ __forceinline__ void load_mma_params(MmaParams& mp, const lcq_pred_params* gp) {
    for (int x = threadIdx.x; x < kNets * 32 * 8; x += blockDim.x) {
        const int net = x >> 8, lane = (x >> 3) & 31, slot = x & 7;
        const int nt = slot >> 2, ks = (slot >> 1) & 1, reg = slot & 1;
        const int n = 8 * nt + (lane >> 2);                      // hidden unit
        const int k = 16 * ks + 2 * (lane & 3) + 8 * reg;        // first of two inputs
        const int8_t* row = &gp->w1[net / 7][net % 7][n][0];
        const int w0 = k < kNin ? row[k] : 0, w1 = k + 1 < kNin ? row[k + 1] : 0;
        mp.bfrag[net][lane][slot] = half_pair(w0, w1);
    }
    const uint32_t r1 = 1u << (gp->s1 - 1);
    for (int x = threadIdx.x; x < kNets * kNhid; x += blockDim.x) {
        const int8_t* row = &gp->w1[x / (7 * kNhid)][(x / kNhid) % 7][x % kNhid][0];
        int32_t wsum = 0;
        for (int t = 0; t < kNin; t++) wsum += row[t];
        (&mp.zk[0][0])[x] = (uint32_t)(&gp->b1[0][0][0])[x] + r1 - 0x4B400000u - 640u * (uint32_t)wsum;
    }
    // W2 as B fragments (rows k = hidden units, column 0 = W2, the other
    // columns 0): lane = 4 g + q holds rows 2q, 2q+1 (reg 0) and 2q+8, 2q+9
    // (reg 1) of column g
    for (int x = threadIdx.x; x < kNets * 32 * 2; x += blockDim.x) {
        const int net = x >> 6, lane = (x >> 1) & 31, reg = x & 1;
        const int g = lane >> 2, k = 2 * (lane & 3) + 8 * reg;
        const int8_t* w2 = &gp->w2[net / 7][net % 7][0];
        mp.w2frag[net][lane][reg] = g == 0 ? half_pair(w2[k], w2[k + 1]) : 0u;
    }
    const uint32_t r2 = 1u << (gp->s2 - 1);
    for (int x = threadIdx.x; x < kNets; x += blockDim.x) {
        const int8_t* w2 = &gp->w2[x / 7][x % 7][0];
        int32_t wsum = 0;
        for (int u = 0; u < kNhid; u++) wsum += w2[u];
        mp.b2k[x] = (uint32_t)(&gp->b2[0][0])[x] + r2 - 1024u * (uint32_t)wsum - 0x4B400000u;
    }
    if (threadIdx.x < 3) mp.s_in[threadIdx.x] = gp->s_in[threadIdx.x];
    if (threadIdx.x == 0) { mp.s1 = gp->s1; mp.s2 = gp->s2; }
}

__device__ __forceinline__ void mma_f16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t a[4], uint32_t saddr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(saddr));
}

// The network output o of the point of this lane (all 32 lanes take part;
// the stencil inputs of the lane's point are already in its row of the
// warp's staging tile `arow`, 32 rows of kArow words).  Both layers run on
// the tensor cores; the first layer's accumulators, turned into the hidden
// values, are the second layer's A fragments without leaving the registers.
__device__ __forceinline__ int32_t network_mma(const MmaParams& mp, int net, const uint32_t* arow) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    uint32_t a[2][2][4];  // [m-tile][k-step]
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(arow);
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const int mtx = lane >> 3, r = lane & 7;
            const int point = 16 * mt + r + 8 * (mtx & 1);
            const int col = 16 * ks + 8 * (mtx >> 1);  // binary16 column
            ldmatrix_x4(a[mt][ks], base + (uint32_t)(point * kArow * 4 + col * 2));
        }
    const int q = lane & 3;
    uint32_t bf[8];
#pragma unroll
    for (int x = 0; x < 8; x++) bf[x] = mp.bfrag[net][lane][x];
    int32_t zk[2][2];  // hidden unit 8 nt + 2 q + e
#pragma unroll
    for (int nt = 0; nt < 2; nt++)
#pragma unroll
        for (int e = 0; e < 2; e++) zk[nt][e] = (int32_t)mp.zk[net][8 * nt + 2 * q + e];
    const uint32_t w2b0 = mp.w2frag[net][lane][0], w2b1 = mp.w2frag[net][lane][1];
    const int s1 = mp.s1;
    // (z >> s1) <= 127 iff z <= hmax; for s1 >= 24 every int32 z >= 0 passes
    const int32_t hmax = s1 >= 24 ? INT_MAX : (int32_t)((128u << s1) - 1u);
    float d[2][4];  // second layer, column 0: the output of each point
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
        float c[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; nt++) {
#pragma unroll
            for (int v = 0; v < 4; v++) c[nt][v] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) mma_f16(c[nt], a[mt][ks], bf[nt * 4 + ks * 2], bf[nt * 4 + ks * 2 + 1]);
        }
        // c[nt][2 hf + e]: point 16 mt + 8 hf + lane / 4, hidden unit 8 nt + 2 q + e.
        // Each accumulator is an integer v = W1 x + 640 sum_t W1[u][t] with
        // |v| <= 27 * 128 * 767 < 2^22, so RN(v + 1.5 2^23) = 1.5 2^23 + v
        // exactly and its bit pattern minus that of 1.5 2^23 is v; with zk,
        // z = W1 x + b1 + 2^(s1-1) (mod 2^32).  h = clamp(z >> s1, 0, 127) =
        // clamp(z, 0, hmax) >> s1, one add-min-max and one shift.  The
        // second layer takes 1024 + h, whose binary16 bit pattern is
        // 0x6400 + h (binary16 values in [1024, 2048) are the integers).
        uint32_t ha[4];  // A fragment: [nt * 2 + hf]
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int hf = 0; hf < 2; hf++) {
                const int32_t z0 = (int32_t)__float_as_uint(__fadd_rn(c[nt][2 * hf], 12582912.0f));
                const int32_t z1 = (int32_t)__float_as_uint(__fadd_rn(c[nt][2 * hf + 1], 12582912.0f));
                const uint32_t h0 = (uint32_t)(__viaddmin_s32_relu(z0, zk[nt][0], hmax) >> s1);
                const uint32_t h1 = (uint32_t)(__viaddmin_s32_relu(z1, zk[nt][1], hmax) >> s1);
                ha[nt * 2 + hf] = 0x64006400u + h0 + (h1 << 16);
            }
#pragma unroll
        for (int v = 0; v < 4; v++) d[mt][v] = 0.0f;
        mma_f16(d[mt], ha, w2b0, w2b1);
    }
    // Column 0 of the output tile sits in the lanes with q = 0: point 16 mt + r
    // in lane 4 (r % 8), register 0 (r < 8) or 2.  Its value is the integer
    // W2 h + 1024 sum_u W2[u], of magnitude below 16 * 128 * 1151 < 2^22, so
    // exact in float32 in any order of the additions.
    const int r = lane & 15, holder = 4 * (r & 7);
    const float v00 = __shfl_sync(0xFFFFFFFFu, d[0][0], holder), v02 = __shfl_sync(0xFFFFFFFFu, d[0][2], holder);
    const float v10 = __shfl_sync(0xFFFFFFFFu, d[1][0], holder), v12 = __shfl_sync(0xFFFFFFFFu, d[1][2], holder);
    const float mine = lane < 16 ? (r < 8 ? v00 : v02) : (r < 8 ? v10 : v12);
    return (int32_t)(__float_as_uint(__fadd_rn(mine, 12582912.0f)) + mp.b2k[net]) >> mp.s2;
}

// The 27 stencil inputs of the point (as in `stencil`) written to the lane's
// row of the staging tile as binary16 pairs of 640 + x_t (x_t = 0 for the
// inputs 27..31, whose weights are 0); returns the
// point's interpolation base (as `interp`) without loads of its own.  The
// interpolation corners are stencil positions: along an axis where the
// point's coordinate x is an odd multiple of s, the floor of x to a multiple
// of 2s is x - s, so positions 1 and 2 are x - s and clamp(x + s), its two
// corners; along an even axis position 1 is x itself.  Summing positions
// {1, 2} of the odd axes and position 1 twice on the even ones adds every
// distinct corner 2^(3 - c) times (c odd axes), so with that sum A the base
// (sum + 2^(c-1)) >> c is (A + 4) >> 3.
__device__ __forceinline__ int32_t stencil_row(const int32_t* p, int N, int i, int j, int k, const Point& pt,
                                               int s_in, uint32_t* row) {
    const int s2 = 2 * pt.s, last = ((N - 1) >> pt.sh) << pt.sh, NN = N * N;
    const int fi = (i >> pt.sh) << pt.sh, fj = (j >> pt.sh) << pt.sh, fk = (k >> pt.sh) << pt.sh;
    int oi[3], oj[3], ok[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        oi[d] = axis_off(clampc(fi + s2 * (d - 1), last), i, NN);
        oj[d] = axis_off(clampc(fj + s2 * (d - 1), last), j, N);
        ok[d] = clampc(fk + s2 * (d - 1), last) - k;
    }
    int32_t c[kNin];
#pragma unroll
    for (int t = 0; t < kNin; t++) c[t] = p[oi[t / 9] + oj[(t / 3) % 3] + ok[t % 3]];
    // interpolation base from positions 1 and 2 (|bins| < 2^30: pairs fit in int32)
    const bool odd_i = pt.cls & 1, odd_j = pt.cls & 2, odd_k = pt.cls & 4;
    long long rj[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        long long rk[2];
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int32_t v1 = c[(a + 1) * 9 + (b + 1) * 3 + 1], v2 = c[(a + 1) * 9 + (b + 1) * 3 + 2];
            rk[b] = (long long)(v1 + (odd_k ? v2 : v1));
        }
        rj[a] = rk[0] + (odd_j ? rk[1] : rk[0]);
    }
    const long long acc = rj[0] + (odd_i ? rj[1] : rj[0]);
    const int32_t base = (int32_t)((acc + 4) >> 3);
    // clamp before the shift: x >> s_in <= 127 iff x <= 128 2^s_in - 1, and
    // >= -128 iff x >= -128 2^s_in (for s_in >= 24 every |x| < 2^31 already
    // shifts into [-128, 127])
    const int32_t lo = s_in >= 24 ? INT_MIN : -(128 << s_in);
    const int32_t hi = s_in >= 24 ? INT_MAX : (128 << s_in) - 1;
    int dv[32];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        if (t < kNin) {
            const int32_t x = __viaddmax_s32(c[t], -base, lo);  // max(c - base, lo); |c|, |base| < 2^30
            dv[t] = (x < hi ? x : hi) >> s_in;
        } else {
            dv[t] = 0;
        }
    }
#pragma unroll
    for (int w = 0; w < 16; w += 4)
        *reinterpret_cast<uint4*>(row + w) = make_uint4(input_pair(dv[2 * w], dv[2 * w + 1]),
                                                        input_pair(dv[2 * w + 2], dv[2 * w + 3]),
                                                        input_pair(dv[2 * w + 4], dv[2 * w + 5]),
                                                        input_pair(dv[2 * w + 6], dv[2 * w + 7]));
    return base;
}

// ---------------------------------------------------------------- kernels --
//
// Interpolation only: one CTA per grid row (i, j) (or lattice row of one
// level when reconstructing), the threads along k, so that every load and
// store of a warp is one coalesced row segment.
//
// With the network, residuals and reconstruction walk each level by boxes
// of coarse cells staged in shared memory (k_net_boxes below).

__global__ void __launch_bounds__(256) k_interp_residuals(const int32_t* __restrict__ bins, int N,
                                                          int32_t* __restrict__ res) {
    const int i = blockIdx.z, j = blockIdx.y;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const size_t e = ((size_t)i * N + j) * N + k;
        const Point pt = classify(i, j, k);
        if (pt.level == 0) {
            res[e] = bins[e];
        } else {
            const int32_t pr = interp_point(bins, N, i, j, k, pt);
            res[e] = (int32_t)((uint32_t)bins[e] - (uint32_t)pr);
        }
    }
}

// The points of one level (anchors when s == 8) on the lattice of multiples of s.
__global__ void __launch_bounds__(256) k_interp_reconstruct(const int32_t* __restrict__ res, int N, int s,
                                                            int32_t* bins) {
    const int i = blockIdx.z * s, j = blockIdx.y * s;
    for (int kk = blockIdx.x * blockDim.x + threadIdx.x; kk * s < N; kk += gridDim.x * blockDim.x) {
        const int k = kk * s;
        const Point pt = classify(i, j, k);
        if (pt.s != s) continue;  // belongs to another level
        const size_t e = ((size_t)i * N + j) * N + k;
        if (pt.level == 0) {
            bins[e] = res[e];
        } else {
            const int32_t pr = interp_point(bins, N, i, j, k, pt);
            bins[e] = (int32_t)((uint32_t)pr + (uint32_t)res[e]);
        }
    }
}

// ------------------------------------------------ boxes of coarse cells --
//
// The network kernels walk each level (stride s, coarse spacing 2s) by boxes
// of coarse cells: cell (ci, cj, ck) is the 2s-cube whose lowest corner is
// the coarse point 2s (ci, cj, ck); it holds the level's point of class
// (a, b, c) at 2s (ci, cj, ck) + s (a, b, c), and that point's stencil is the
// coarse points of cells ci-1..ci+1 (and likewise along j, k), each index
// clamped to [0, L], L = last / 2s.  A CTA copies a box's coarse points,
// clamped, with a halo of one cell on every side, into shared memory once
// (BI x BJ x BK cells: (BI+2)(BJ+2)(BK+2) values); then each warp takes the
// 32 cells of one box row along k for one class, so that every stencil input
// is a shared-memory load at a fixed offset from the lane's cell and the 32
// lanes share the class and the network.  Persistent CTAs load the network
// parameters once.
constexpr int kBI = 2, kBJ = 4, kBK = 32;
constexpr int kHI = kBI + 2, kHJ = kBJ + 2, kHK = kBK + 2;
constexpr int kHalo = kHI * kHJ * kHK;

struct BoxLevel {
    int s, sh, L;          // stride, log2(2s), largest coarse index
    int nb[3];             // boxes along i, j, k
    uint32_t first_box;    // boxes of the levels before this one in the launch
};

struct BoxTable {
    BoxLevel lv[3];
    int count;
    uint32_t total;
};

// The levels of one launch: level > 0 that level only, -1 levels 1..3.
static BoxTable box_table(int N, int level) {
    BoxTable t{};
    uint32_t boxes = 0;
    for (int l = 1; l <= 3; l++) {
        if (level > 0 && level != l) continue;
        BoxLevel& B = t.lv[t.count++];
        B.s = 8 >> l;
        B.sh = 4 - l;  // log2(2s)
        const int last = ((N - 1) >> B.sh) << B.sh;
        B.L = last >> B.sh;
        const int cells = B.L + 1;
        B.nb[0] = (cells + kBI - 1) / kBI;
        B.nb[1] = (cells + kBJ - 1) / kBJ;
        B.nb[2] = (cells + kBK - 1) / kBK;
        B.first_box = boxes;
        boxes += (uint32_t)B.nb[0] * B.nb[1] * B.nb[2];
    }
    t.total = boxes;
    return t;
}

// The base and the 27 stencil inputs of a point from its coarse bins c[t],
// t = 9 di + 3 dj + dk (d = 0, 1, 2 for the cells before, at and after the
// point's own), written to the lane's row of the warp's staging tile as in
// stencil_row; returns the interpolation base.
__device__ __forceinline__ int32_t stencil_inputs(const int32_t c[kNin], int cls, int s_in, uint32_t* row) {
    const bool odd_i = cls & 1, odd_j = cls & 2, odd_k = cls & 4;
    long long rj[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        long long rk[2];
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int32_t v1 = c[(a + 1) * 9 + (b + 1) * 3 + 1], v2 = c[(a + 1) * 9 + (b + 1) * 3 + 2];
            rk[b] = (long long)(v1 + (odd_k ? v2 : v1));
        }
        rj[a] = rk[0] + (odd_j ? rk[1] : rk[0]);
    }
    const long long acc = rj[0] + (odd_i ? rj[1] : rj[0]);
    const int32_t base = (int32_t)((acc + 4) >> 3);
    // clamp before the shift (as in stencil_row): one add-max, one min, one shift
    const int32_t lo = s_in >= 24 ? INT_MIN : -(128 << s_in);
    const int32_t hi = s_in >= 24 ? INT_MAX : (128 << s_in) - 1;
    int dv[32];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        if (t < kNin) {
            const int32_t x = __viaddmax_s32(c[t], -base, lo);  // max(c - base, lo); |c|, |base| < 2^30
            dv[t] = (x < hi ? x : hi) >> s_in;
        } else {
            dv[t] = 0;
        }
    }
#pragma unroll
    for (int w = 0; w < 16; w += 4)
        *reinterpret_cast<uint4*>(row + w) = make_uint4(input_pair(dv[2 * w], dv[2 * w + 1]),
                                                        input_pair(dv[2 * w + 2], dv[2 * w + 3]),
                                                        input_pair(dv[2 * w + 4], dv[2 * w + 5]),
                                                        input_pair(dv[2 * w + 6], dv[2 * w + 7]));
    return base;
}

// RECON = false: res = bins - prediction for the levels of the table.
// RECON = true: bins = prediction + res for one level, whose predictions
// read only coarser levels, already reconstructed (anchors by k_anchors).
// Warp w of the CTA takes jobs w, w + 8, ...: job = (class - 1) * 8 + box row.
struct NetSmem {
    MmaParams mp;
    alignas(16) uint32_t a[8][32 * kArow];  // per-warp staging tiles (16-byte rows: vector stores, ldmatrix)
    int32_t halo[kHalo];
};
static_assert(offsetof(NetSmem, a) % 16 == 0 && (kArow * 4) % 16 == 0, "16-byte aligned staging rows");

template <bool RECON>
__global__ void __launch_bounds__(256) k_net_boxes(const int32_t* __restrict__ in, int N,
                                                   const lcq_pred_params* params, int32_t* out, const BoxTable bt) {
    extern __shared__ __align__(16) unsigned char net_smem[];
    NetSmem& S = *reinterpret_cast<NetSmem*>(net_smem);
    load_mma_params(S.mp, params);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* arow = &S.a[warp][0];
    const int32_t* src = RECON ? out : in;  // where the coarse bins are read
    const size_t NN = (size_t)N * N;
    int l = 0;  // boxes only grow, so the level search resumes where it stopped
    for (uint32_t box = blockIdx.x; box < bt.total; box += gridDim.x) {
        while (l + 1 < bt.count && box >= bt.lv[l + 1].first_box) l++;
        const BoxLevel& B = bt.lv[l];
        const uint32_t r = box - B.first_box;
        const int bk = (int)(r % (uint32_t)B.nb[2]);
        const int bj = (int)((r / (uint32_t)B.nb[2]) % (uint32_t)B.nb[1]);
        const int bi = (int)(r / ((uint32_t)B.nb[2] * (uint32_t)B.nb[1]));
        const int ci0 = bi * kBI, cj0 = bj * kBJ, ck0 = bk * kBK;
        __syncthreads();  // the previous box's halo is no longer read (and the parameters are loaded)
        for (int x = threadIdx.x; x < kHalo; x += blockDim.x) {
            const int hk = x % kHK, hj = (x / kHK) % kHJ, hi = x / (kHK * kHJ);
            const int ci = clampc(ci0 - 1 + hi, B.L), cj = clampc(cj0 - 1 + hj, B.L), ck = clampc(ck0 - 1 + hk, B.L);
            S.halo[x] = src[((size_t)(ci << B.sh) * N + (size_t)(cj << B.sh)) * N + (size_t)(ck << B.sh)];
        }
        __syncthreads();
        const int s = B.s, net0 = (3 - B.sh) * 7;  // level - 1 = 3 - sh
        const int s_in = S.mp.s_in[3 - B.sh];
        for (int job = warp; job < 7 * kBI * kBJ; job += 8) {
            const int cls = job / (kBI * kBJ) + 1, row = job % (kBI * kBJ);
            const int ri = row / kBJ, rj = row % kBJ;
            const int i = ((ci0 + ri) << B.sh) + ((cls & 1) ? s : 0);
            const int j = ((cj0 + rj) << B.sh) + ((cls & 2) ? s : 0);
            const int k = ((ck0 + lane) << B.sh) + ((cls & 4) ? s : 0);
            const bool valid = i < N && j < N && k < N;
            const int32_t* h = &S.halo[((ri + 1) * kHJ + (rj + 1)) * kHK + lane + 1];
            int32_t c[kNin];
#pragma unroll
            for (int t = 0; t < kNin; t++) c[t] = h[(t / 9 - 1) * kHJ * kHK + ((t / 3) % 3 - 1) * kHK + (t % 3 - 1)];
            const int32_t base = stencil_inputs(c, cls, s_in, arow + lane * kArow);
            const int32_t pr = (int32_t)((uint32_t)base + (uint32_t)network_mma(S.mp, net0 + cls - 1, arow));
            __syncwarp();  // the staging tile is rewritten by the next job
            if (valid) {
                const size_t e = (size_t)i * NN + (size_t)j * N + (size_t)k;
                out[e] = RECON ? (int32_t)((uint32_t)pr + (uint32_t)in[e]) : (int32_t)((uint32_t)in[e] - (uint32_t)pr);
            }
        }
    }
}

// Anchors (all coordinates multiples of 8) are kept as they are.
__global__ void __launch_bounds__(256) k_anchors(const int32_t* __restrict__ in, int N, int32_t* __restrict__ out) {
    const int m = (N + 7) / 8;
    const uint32_t total = (uint32_t)m * m * m;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
        const int k = (int)(x % m) * 8, j = (int)((x / m) % m) * 8, i = (int)(x / ((uint32_t)m * m)) * 8;
        const size_t e = ((size_t)i * N + j) * N + k;
        out[e] = in[e];
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

// Launch of k_net_boxes: a persistent grid of the CTAs that fit on the
// device at once, at most one per box, with the shared-memory opt-in made
// once per device.
template <bool RECON>
static cudaError_t launch_net_boxes(const int32_t* in, int N, const lcq_pred_params* params, int32_t* out,
                                    const BoxTable& bt, cudaStream_t stream) {
    static lcq::OccupancyCache cache{};
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = lcq::cached_blocks_per_sm(cache, dev, k_net_boxes<RECON>, 256, sizeof(NetSmem));
    uint64_t g = (uint64_t)per_sm * (uint64_t)(sms > 0 ? sms : 148);
    if (g > bt.total) g = bt.total;
    if (g < 1) g = 1;
    k_net_boxes<RECON><<<(unsigned)g, 256, sizeof(NetSmem), stream>>>(in, N, params, out, bt);
    return cudaPeekAtLastError();
}

}  // namespace pred
}  // namespace lcq

using namespace lcq::pred;

extern "C" {

lcq_status lcq_pred_residuals(const int32_t* d_bins, uint32_t N, const lcq_pred_params* d_params, int32_t* d_res,
                              cudaStream_t stream) {
    if (!n_ok((int)N) || !d_bins || !d_res) return LCQ_ERR_ARG;
    if (d_params) {
        const BoxTable bt = box_table((int)N, -1);
        const uint32_t m = (N + 7) / 8;
        k_anchors<<<(m * m * m + 255) / 256, 256, 0, stream>>>(d_bins, (int)N, d_res);
        if (launch_net_boxes<false>(d_bins, (int)N, d_params, d_res, bt, stream) != cudaSuccess) return LCQ_ERR_CUDA;
    } else {
        const dim3 grid((N + 255) / 256, N, N);
        k_interp_residuals<<<grid, 256, 0, stream>>>(d_bins, (int)N, d_res);
    }
    return cudaPeekAtLastError() == cudaSuccess ? LCQ_OK : LCQ_ERR_CUDA;
}

lcq_status lcq_pred_reconstruct(const int32_t* d_res, uint32_t N, const lcq_pred_params* d_params, int32_t* d_bins,
                                cudaStream_t stream) {
    if (!n_ok((int)N) || !d_bins || !d_res) return LCQ_ERR_ARG;
    for (int level = 0; level <= 3; level++) {
        if (d_params && level == 0) {
            const uint32_t m = (N + 7) / 8;
            k_anchors<<<(m * m * m + 255) / 256, 256, 0, stream>>>(d_res, (int)N, d_bins);
        } else if (d_params) {
            const BoxTable bt = box_table((int)N, level);
            if (launch_net_boxes<true>(d_res, (int)N, d_params, d_bins, bt, stream) != cudaSuccess) return LCQ_ERR_CUDA;
        } else {
            const int s = 8 >> level;
            const unsigned m = (N + s - 1) / s;
            const dim3 grid((m + 255) / 256, m, m);
            k_interp_reconstruct<<<grid, 256, 0, stream>>>(d_res, (int)N, s, d_bins);
        }
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
    static lcq::OccupancyCache opt_in{};  // the shared-memory opt-in, once per device
    int dev = 0;
    cudaGetDevice(&dev);
    lcq::cached_blocks_per_sm(opt_in, dev, k_train_partial, kTrainBlock, smem);
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
