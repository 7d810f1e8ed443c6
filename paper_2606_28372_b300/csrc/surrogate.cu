// MLP surrogate that screens an oversampled proposal pool (not part of the paper's
// method; the constraint-aware optimizer stays its fallback and judge).
//
// Network: one-hot value indices (D = sum_k r_k features, one active per
// parameter) -> H -> H -> H (ReLU) -> 1.  Masters are fp32; the forward and
// backward passes use bf16(W) (round to nearest even) and accumulate in fp32
// with one fused multiply-add per term in ascending index order, on CUDA cores,
// so predictions, gradients and updates are reproducible bit for bit.  Loss:
// mean squared error against log-fitness; SGD with momentum.
//
// A screened generation of DE or GA proposes `pool` candidates per slot
// (RNG streams offset by the pool index), repairs all of them exactly, applies
// the GA mutation, predicts all, keeps the lowest prediction per slot (ties:
// smaller key, then smaller pool index) and evaluates only those.  Every
// generation the surrogate is judged on what was evaluated (mean absolute error
// of its predictions, made before it learns from them) and trained on batches
// drawn from everything evaluated so far.  Screening is on only after
// warmup_mult * pop evaluations and while the error is at most mae_ratio times
// the mean absolute deviation of the generation's log-fitness.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "internal.hpp"
#include "optim_dev.cuh"

namespace ct {
ct_status evaluate_impl(ct_space* s, uint32_t* memo, unsigned long long* unique, unsigned long long* cost_acc,
                        const uint64_t* d_keys, int64_t n, float* d_fit, int64_t* d_rank, cudaStream_t st,
                        float invalid_fit = __builtin_inff());

__device__ __forceinline__ float bf16r(float f) {
    uint32_t u = __float_as_uint(f);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xFFFF0000u);
}

struct MlpOff {
    size_t W1, b1, W2, b2, W3, b3, W4, b4, total;
};

static MlpOff mlp_off(int D, int H) {
    MlpOff o;
    o.W1 = 0;
    o.b1 = o.W1 + (size_t)H * D;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (size_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + (size_t)H * H;
    o.W4 = o.b3 + H;
    o.b4 = o.W4 + H;
    o.total = o.b4 + 1;
    return o;
}

// ------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------
// Glorot-uniform weights from the MLP_INIT stream (individual = tensor 1..4, word =
// element index), zero biases.
__global__ void k_mlp_init(float* __restrict__ p, MlpOff o, uint64_t seed, float a1, float a2, float a3, float a4) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < o.total; e += (size_t)gridDim.x * blockDim.x) {
        int t = 0;
        size_t local = 0;
        float a = 0.0f;
        if (e < o.b1) { t = 1; local = e - o.W1; a = a1; }
        else if (e >= o.W2 && e < o.b2) { t = 2; local = e - o.W2; a = a2; }
        else if (e >= o.W3 && e < o.b3) { t = 3; local = e - o.W3; a = a3; }
        else if (e >= o.W4 && e < o.b4) { t = 4; local = e - o.W4; a = a4; }
        float v = 0.0f;
        if (t) {
            const float u = u01(rng_word(seed, (uint32_t)t, 0, PU_MLP_INIT, (uint32_t)local));
            v = __fmul_rn(__fsub_rn(__fmul_rn(2.0f, u), 1.0f), a);
        }
        p[e] = v;
    }
}

// one-hot feature indices of keys: base_k + index of parameter k
__global__ void k_feats(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ keys, int B,
                        int32_t* __restrict__ feats) {
    const int N = sp->n;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const uint64_t key = keys[b];
        int base = 0;
        for (int k = 0; k < N; ++k) {
            feats[(size_t)b * N + k] = base + field(sp, key, k);
            base += sp->r[k];
        }
    }
}

// layer 1 on the one-hot input: z = (sum of the active bf16 weights, ascending) + b
__global__ void k_mlp_l1(const float* __restrict__ p, MlpOff o, int D, int H, int N, const int32_t* __restrict__ feats,
                         int B, float* __restrict__ z, float* __restrict__ h) {
    const size_t total = (size_t)B * H;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(g / H), j = (int)(g % H);
        const int32_t* f = feats + (size_t)b * N;
        float acc = 0.0f;
        for (int k = 0; k < N; ++k) acc = __fadd_rn(acc, bf16r(p[o.W1 + (size_t)j * D + f[k]]));
        const float zz = __fadd_rn(acc, p[o.b1 + j]);
        z[g] = zz;
        h[g] = zz > 0.0f ? zz : 0.0f;
    }
}

// Ordered product C[m][n] = sum_{k ascending} A(m,k) * Bv(n,k), one fused multiply-add per
// term starting from 0, A(m,k) = A[m*sam + k*sak], Bv(n,k) = B[n*sbn + k*sbk] (optionally
// bf16-rounded).  One output per thread in tiles of OG_T x OG_T outputs (256 CTAs for a
// 256 x 256 product, more than the SMs: every output is one sequential chain of K terms, so the
// products of the training steps are latency-bound and want many threads), k in chunks of OG_K
// through shared memory; the next chunk's elements are loaded into registers while the current
// chunk is multiplied.
// EPI 0: z = acc + bias[n] -> out (z) and out2 (ReLU);  EPI 1: out = zmask > 0 ? acc : 0;
// EPI 2: out = acc (and, with rowsum, rowsum[m] = sum_{k ascending} A(m,k), added from 0: the
// bias gradients, by the threads of column 0);  EPI 3: out = acc + bias[n].
constexpr int OG_T = 16, OG_K = 64, OG_THREADS = OG_T * OG_T, OG_PER = OG_T * OG_K / OG_THREADS;

// One product's arguments (see k_ogemm).
struct OgArgs {
    int M, Nn, K;
    const float* A;
    long sam, sak;
    const float* Bm;
    long sbn, sbk;
    const float* bias;
    const float* zmask;
    float* out;
    float* out2;
    long ldc;
    float* rowsum;
};

// The output tile (bx, by) of one ordered product.
template <int EPI, bool BF16>
__device__ __forceinline__ void ogemm_tile(const OgArgs& g, int bx, int by) {
    const int M = g.M, Nn = g.Nn, K = g.K;
    const float* __restrict__ A = g.A;
    const float* __restrict__ Bm = g.Bm;
    const long sam = g.sam, sak = g.sak, sbn = g.sbn, sbk = g.sbk, ldc = g.ldc;
    const float* __restrict__ bias = g.bias;
    const float* __restrict__ zmask = g.zmask;
    float* __restrict__ out = g.out;
    float* __restrict__ out2 = g.out2;
    float* __restrict__ rowsum = g.rowsum;
    __shared__ float As[OG_T][OG_K + 1], Bs[OG_T][OG_K + 1];
    const int tx = threadIdx.x % OG_T, ty = threadIdx.x / OG_T;
    const int m0 = by * OG_T, n0 = bx * OG_T;
    const bool do_rs = EPI == 2 && rowsum && bx == 0 && tx == 0;
    // the elements this thread stages, e = threadIdx.x + q * OG_THREADS: consecutive threads run
    // along the operand's unit stride (k for a row-major operand, the row otherwise), so that the
    // loads are contiguous; the shared rows are padded, so either order stores without conflicts
    const bool ak = sak == 1, bk = sbk == 1;
    auto rc = [](bool along_k, int e, int& r, int& c) {
        if (along_k) { r = e / OG_K; c = e % OG_K; } else { r = e % OG_T; c = e / OG_T; }
    };
    float pa[OG_PER], pb[OG_PER];
    auto fetch = [&](int k0) {
        const int kmax = min(OG_K, K - k0);
#pragma unroll
        for (int q = 0; q < OG_PER; ++q) {
            const int e = threadIdx.x + q * OG_THREADS;
            int r, c;
            rc(ak, e, r, c);
            const int m = m0 + r;
            pa[q] = (m < M && c < kmax) ? A[m * sam + (k0 + c) * sak] : 0.0f;
            rc(bk, e, r, c);
            const int n = n0 + r;
            const float bv = (n < Nn && c < kmax) ? Bm[n * sbn + (k0 + c) * sbk] : 0.0f;
            pb[q] = BF16 ? bf16r(bv) : bv;
        }
    };
    fetch(0);
    float acc = 0.0f, rs = 0.0f;
    for (int k0 = 0; k0 < K; k0 += OG_K) {
        const int kmax = min(OG_K, K - k0);
#pragma unroll
        for (int q = 0; q < OG_PER; ++q) {
            const int e = threadIdx.x + q * OG_THREADS;
            int r, c;
            rc(ak, e, r, c);
            As[r][c] = pa[q];
            rc(bk, e, r, c);
            Bs[r][c] = pb[q];
        }
        __syncthreads();
        if (k0 + OG_K < K) fetch(k0 + OG_K);   // in flight while this chunk is multiplied
        for (int kk = 0; kk < kmax; ++kk) {
            acc = __fmaf_rn(As[ty][kk], Bs[tx][kk], acc);
            if (do_rs) rs = __fadd_rn(rs, As[ty][kk]);
        }
        __syncthreads();
    }
    const int m = m0 + ty, n = n0 + tx;
    if (do_rs && m < M) rowsum[m] = rs;
    if (m >= M || n >= Nn) return;
    const long idx = m * ldc + n;
    if (EPI == 0) {
        const float z = __fadd_rn(acc, bias[n]);
        out[idx] = z;
        out2[idx] = z > 0.0f ? z : 0.0f;
    } else if (EPI == 1) {
        out[idx] = zmask[idx] > 0.0f ? acc : 0.0f;
    } else if (EPI == 2) {
        out[idx] = acc;
    } else {
        out[idx] = __fadd_rn(acc, bias[n]);
    }
}


template <int EPI, bool BF16>
__global__ void __launch_bounds__(OG_THREADS)
k_ogemm(int M, int Nn, int K, const float* __restrict__ A, long sam, long sak, const float* __restrict__ Bm, long sbn,
        long sbk, const float* __restrict__ bias, const float* __restrict__ zmask, float* __restrict__ out,
        float* __restrict__ out2, long ldc, float* __restrict__ rowsum) {
    const OgArgs g{M, Nn, K, A, sam, sak, Bm, sbn, sbk, bias, zmask, out, out2, ldc, rowsum};
    ogemm_tile<EPI, BF16>(g, blockIdx.x, blockIdx.y);
}

// The backward products that do not wait for one another, in one launch (blockIdx.z picks the
// product; each keeps its own tiles): the delta through a layer's weights (EPI 1, bf16 weights)
// beside the weight gradients (EPI 2) that need only the deltas already computed.  Each output
// is computed exactly as by k_ogemm.
__global__ void __launch_bounds__(OG_THREADS)
k_ogemm_bwd(const OgArgs dl, const OgArgs gw0, const OgArgs gw1, int n_gw) {
    const int z = blockIdx.z;
    if (z == 0) {
        if ((int)blockIdx.x * OG_T < dl.Nn && (int)blockIdx.y * OG_T < dl.M) ogemm_tile<1, true>(dl, blockIdx.x, blockIdx.y);
    } else {
        const OgArgs& g = z == 1 ? gw0 : gw1;
        if (z <= n_gw && (int)blockIdx.x * OG_T < g.Nn && (int)blockIdx.y * OG_T < g.M)
            ogemm_tile<2, false>(g, blockIdx.x, blockIdx.y);
    }
}

// The same ordered product for tall products (the screening pool's forward pass): a CTA of 64
// threads computes a 32 x 32 tile, 4 x 4 outputs per thread in registers, so each pair of
// 16-byte shared loads feeds 16 fused multiply-adds; tiles are staged k-major (rows padded to
// 36 floats, four consecutive rows per 16-byte store).  Each output still takes its terms one at
// a time in ascending k from 0, so it equals k_ogemm's bit for bit.  EPI 0 and 3 as above.
constexpr int O4_T = 32, O4_K = 32, O4_R = 4, O4_THREADS = (O4_T / O4_R) * (O4_T / O4_R), O4_LD = O4_T + 4;
constexpr int O4_MIN_ROWS = 1024;   // forward passes of at least this many samples take k_ogemm4

constexpr int O4_PER = O4_K * (O4_T / 4) / O4_THREADS;   // 16-byte groups a thread stages per operand

// One operand's chunk into registers (all loads issued before any is used), then into shared
// memory: group e = threadIdx.x + q * O4_THREADS holds X(r0 + 4 g .. + 3, k0 + c); the lanes run
// along the operand's unit stride.
__device__ __forceinline__ void o4_coords(long sk, int e, int& c, int& g) {
    if (sk == 1) { c = e % O4_K; g = e / O4_K; } else { g = e % (O4_T / 4); c = e / (O4_T / 4); }
}
template <bool BF16>
__device__ __forceinline__ void o4_load(float (&v)[O4_PER][4], const float* __restrict__ X, long sr, long sk, int rows,
                                        int r0, int k0, int kmax) {
#pragma unroll
    for (int q = 0; q < O4_PER; ++q) {
        int c, g;
        o4_coords(sk, threadIdx.x + q * O4_THREADS, c, g);
        const int r = r0 + 4 * g;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = (c < kmax && r + i < rows) ? X[(long)(r + i) * sr + (long)(k0 + c) * sk] : 0.0f;
            v[q][i] = BF16 ? bf16r(x) : x;
        }
    }
}
__device__ __forceinline__ void o4_store(float (*S)[O4_LD], const float (&v)[O4_PER][4], long sk) {
#pragma unroll
    for (int q = 0; q < O4_PER; ++q) {
        int c, g;
        o4_coords(sk, threadIdx.x + q * O4_THREADS, c, g);
        *reinterpret_cast<float4*>(&S[c][4 * g]) = make_float4(v[q][0], v[q][1], v[q][2], v[q][3]);
    }
}

template <int EPI, bool BF16>
__global__ void __launch_bounds__(O4_THREADS)
k_ogemm4(int M, int Nn, int K, const float* __restrict__ A, long sam, long sak, const float* __restrict__ Bm, long sbn,
         long sbk, const float* __restrict__ bias, float* __restrict__ out, float* __restrict__ out2, long ldc) {
    __shared__ __align__(16) float As[O4_K][O4_LD], Bs[O4_K][O4_LD];
    const int tx = threadIdx.x % (O4_T / O4_R), ty = threadIdx.x / (O4_T / O4_R);
    const int m0 = blockIdx.y * O4_T, n0 = blockIdx.x * O4_T;
    float acc[O4_R][O4_R];
#pragma unroll
    for (int i = 0; i < O4_R; ++i)
#pragma unroll
        for (int j = 0; j < O4_R; ++j) acc[i][j] = 0.0f;
    float va[O4_PER][4], vb[O4_PER][4];
    o4_load<false>(va, A, sam, sak, M, m0, 0, min(O4_K, K));
    o4_load<BF16>(vb, Bm, sbn, sbk, Nn, n0, 0, min(O4_K, K));
    for (int k0 = 0; k0 < K; k0 += O4_K) {
        const int kmax = min(O4_K, K - k0);
        o4_store(As, va, sak);
        o4_store(Bs, vb, sbk);
        __syncthreads();
        if (k0 + O4_K < K) {   // the next chunk is in flight while this one is multiplied
            o4_load<false>(va, A, sam, sak, M, m0, k0 + O4_K, min(O4_K, K - k0 - O4_K));
            o4_load<BF16>(vb, Bm, sbn, sbk, Nn, n0, k0 + O4_K, min(O4_K, K - k0 - O4_K));
        }
        for (int kk = 0; kk < kmax; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * O4_R]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * O4_R]);
            const float av[O4_R] = {a4.x, a4.y, a4.z, a4.w}, bv[O4_R] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int i = 0; i < O4_R; ++i)
#pragma unroll
                for (int j = 0; j < O4_R; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < O4_R; ++i) {
        const int m = m0 + ty * O4_R + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < O4_R; ++j) {
            const int n = n0 + tx * O4_R + j;
            if (n >= Nn) continue;
            const long idx = m * ldc + n;
            const float z = __fadd_rn(acc[i][j], bias[n]);
            out[idx] = z;
            if (EPI == 0) out2[idx] = z > 0.0f ? z : 0.0f;
        }
    }
}

static dim3 og_grid(int M, int Nn) { return dim3((Nn + OG_T - 1) / OG_T, (M + OG_T - 1) / OG_T); }

// output gradient and the last hidden layer's delta
__global__ void k_mlp_gout(const float* __restrict__ pred, const float* __restrict__ y, int B, float scale,
                           float* __restrict__ gout) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) gout[b] = __fmul_rn(scale, __fsub_rn(pred[b], y[b]));
}

__global__ void k_mlp_d3(const float* __restrict__ p, MlpOff o, int H, int B, const float* __restrict__ gout,
                         const float* __restrict__ z3, float* __restrict__ d3) {
    const size_t total = (size_t)B * H;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(g / H), j = (int)(g % H);
        d3[g] = z3[g] > 0.0f ? __fmul_rn(gout[b], bf16r(p[o.W4 + j])) : 0.0f;
    }
}

// Gradient of the one-hot layer and of its bias.  A CTA takes JB hidden units; thread (jj, k)
// owns the outputs gW1[j][base_k .. base_k + r_k) of parameter k's values (kept in shared memory,
// no other thread writes them) and adds d1[b][j] to the one that sample b activates, in
// ascending b; thread (jj, 0) also sums d1[b][j] over b for the bias.  Every output is thus its
// plain ascending-sample sum from 0 (features never active stay 0).  Samples are staged through
// shared memory in chunks of W1_CHUNK.
constexpr int W1_CHUNK = 256;

static __host__ __device__ size_t w1grad_ft_off(int JB, int D) {   // floats before the feature tile (16-byte aligned)
    return ((size_t)JB * D + (size_t)W1_CHUNK * JB + 3) & ~(size_t)3;
}
static size_t w1grad_smem(int JB, int D, int N) {
    return (w1grad_ft_off(JB, D) + (size_t)W1_CHUNK * N) * sizeof(float);
}

__global__ void k_mlp_w1grad(const float* __restrict__ d1, const int32_t* __restrict__ feats, int B, int N, int D,
                             int H, int JB, float* __restrict__ gW1, float* __restrict__ gb1) {
    extern __shared__ __align__(16) float w1s[];
    float* outs = w1s;                                        // [JB][D]
    float* dt = outs + (size_t)JB * D;                        // [W1_CHUNK][JB]
    int32_t* ft = reinterpret_cast<int32_t*>(w1s + w1grad_ft_off(JB, D));   // [W1_CHUNK][N]
    const int j0 = blockIdx.x * JB;
    const int t = threadIdx.x, jj = t / N, k = t % N;
    const bool mine = jj < JB && j0 + jj < H;
    for (int e = t; e < JB * D; e += blockDim.x) outs[e] = 0.0f;
    float bsum = 0.0f;
    for (int b0 = 0; b0 < B; b0 += W1_CHUNK) {
        const int nb = min(W1_CHUNK, B - b0);
        __syncthreads();   // the previous chunk is done with dt and ft (and outs is zeroed)
        // eight loads in flight per thread before their stores
        for (int e0 = t; e0 < nb * JB; e0 += 8 * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * blockDim.x, bb = e / JB, q = e % JB;
                v[u] = (e < nb * JB && j0 + q < H) ? d1[(size_t)(b0 + bb) * H + j0 + q] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (e0 + u * (int)blockDim.x < nb * JB) dt[e0 + u * blockDim.x] = v[u];
        }
        if ((N & 3) == 0) {   // 16-byte loads of the sample rows
            const int4* src = reinterpret_cast<const int4*>(feats + (size_t)b0 * N);
            int4* dst = reinterpret_cast<int4*>(ft);
            const int nv4 = nb * N / 4;
            for (int e0 = t; e0 < nv4; e0 += 8 * blockDim.x) {
                int4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e0 + u * (int)blockDim.x < nv4) v[u] = src[e0 + u * blockDim.x];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (e0 + u * (int)blockDim.x < nv4) dst[e0 + u * blockDim.x] = v[u];
            }
        } else {
            for (int e = t; e < nb * N; e += blockDim.x) ft[e] = feats[(size_t)b0 * N + e];
        }
        __syncthreads();
        if (mine) {
            float* row = outs + (size_t)jj * D;
            for (int bb = 0; bb < nb; ++bb) {
                const float v = dt[bb * JB + jj];
                const int f = ft[bb * N + k];
                row[f] = __fadd_rn(row[f], v);
                if (k == 0) bsum = __fadd_rn(bsum, v);
            }
        }
    }
    __syncthreads();
    for (int e = t; e < JB * D; e += blockDim.x) {
        const int q = e / D, f = e % D;
        if (j0 + q < H) gW1[(size_t)(j0 + q) * D + f] = outs[e];
    }
    if (mine && k == 0) gb1[j0 + jj] = bsum;
}

// The same gradient for inputs too wide for the shared-memory form: one thread per (j, feature f)
// sums d1[b][j] over the samples (ascending) in which f is active; an owner index outside 0..N-1
// means f is never active.  The bias is left to k_colsum.
__global__ void k_mlp_w1grad_wide(const float* __restrict__ d1, const int32_t* __restrict__ feats,
                                  const int32_t* __restrict__ param_of, int B, int N, int D, int H,
                                  float* __restrict__ gW1) {
    const size_t total = (size_t)H * D;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(g / D), f = (int)(g % D);
        const int k = param_of[f];
        float acc = 0.0f;
        if (k >= 0 && k < N)
            for (int b = 0; b < B; ++b)
                if (feats[(size_t)b * N + k] == f) acc = __fadd_rn(acc, d1[(size_t)b * H + j]);
        gW1[g] = acc;
    }
}

// column sums over the batch in ascending sample order
__global__ void k_colsum(const float* __restrict__ d, int cols, int B, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float acc = 0.0f;
    for (int b = 0; b < B; ++b) acc = __fadd_rn(acc, d[(size_t)b * cols + j]);
    out[j] = acc;
}

__global__ void k_mlp_sgd(float* __restrict__ p, float* __restrict__ mom, const float* __restrict__ g, size_t n, float lr,
                          float mu) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float v = __fadd_rn(__fmul_rn(mu, mom[e]), g[e]);
        mom[e] = v;
        p[e] = __fsub_rn(p[e], __fmul_rn(lr, v));
    }
}

// ------------------------------------------------------------------------------
// host: forward / gradient drivers over a workspace
// ------------------------------------------------------------------------------
struct MlpWork {       // floats, each [n x H] unless noted
    float *z1, *h1, *z2, *h2, *z3, *h3, *d1, *d2, *d3, *gout;
};

static size_t work_floats(int H, int B) { return (size_t)B * H * 9 + (size_t)B; }

static MlpWork carve(float* w, int H, int B) {
    MlpWork m;
    const size_t s = (size_t)B * H;
    m.z1 = w; m.h1 = w + s; m.z2 = w + 2 * s; m.h2 = w + 3 * s; m.z3 = w + 4 * s; m.h3 = w + 5 * s;
    m.d1 = w + 6 * s; m.d2 = w + 7 * s; m.d3 = w + 8 * s; m.gout = w + 9 * s;
    return m;
}

static unsigned grid_for(size_t n, int threads = 256) { return (unsigned)std::min<size_t>((n + threads - 1) / threads, 148 * 16); }

static ct_status mlp_forward_impl(const float* p, int D, int H, int N, const int32_t* feats, int B, float* pred,
                                  const MlpWork& w, cudaStream_t st) {
    const MlpOff o = mlp_off(D, H);
    k_mlp_l1<<<grid_for((size_t)B * H), 256, 0, st>>>(p, o, D, H, N, feats, B, w.z1, w.h1);
    if (B >= O4_MIN_ROWS) {   // tall: register-blocked tiles
        const dim3 g4((H + O4_T - 1) / O4_T, (B + O4_T - 1) / O4_T);
        k_ogemm4<0, true><<<g4, O4_THREADS, 0, st>>>(B, H, H, w.h1, H, 1, p + o.W2, H, 1, p + o.b2, w.z2, w.h2, H);
        k_ogemm4<0, true><<<g4, O4_THREADS, 0, st>>>(B, H, H, w.h2, H, 1, p + o.W3, H, 1, p + o.b3, w.z3, w.h3, H);
        k_ogemm<3, true><<<og_grid(B, 1), OG_THREADS, 0, st>>>(B, 1, H, w.h3, H, 1, p + o.W4, 0, 1, p + o.b4, nullptr,
                                                               pred, nullptr, 1, nullptr);
        count_launch(4);
        CT_TRY_CUDA(cudaGetLastError());
        return CT_OK;
    }
    const dim3 g = og_grid(B, H);
    k_ogemm<0, true><<<g, OG_THREADS, 0, st>>>(B, H, H, w.h1, H, 1, p + o.W2, H, 1, p + o.b2, nullptr, w.z2, w.h2, H,
                                               nullptr);
    k_ogemm<0, true><<<g, OG_THREADS, 0, st>>>(B, H, H, w.h2, H, 1, p + o.W3, H, 1, p + o.b3, nullptr, w.z3, w.h3, H,
                                               nullptr);
    k_ogemm<3, true><<<og_grid(B, 1), OG_THREADS, 0, st>>>(B, 1, H, w.h3, H, 1, p + o.W4, 0, 1, p + o.b4, nullptr,
                                                           pred, nullptr, 1, nullptr);
    count_launch(4);
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

static ct_status mlp_grad_impl(const float* p, int D, int H, int N, const int32_t* feats, const float* y, int B,
                               float* grad, float* pred, const int32_t* param_of, const MlpWork& w, cudaStream_t st) {
    const MlpOff o = mlp_off(D, H);
    CT_TRY(mlp_forward_impl(p, D, H, N, feats, B, pred, w, st));
    const float scale = 2.0f / (float)B;
    k_mlp_gout<<<(B + 255) / 256, 256, 0, st>>>(pred, y, B, scale, w.gout);
    k_mlp_d3<<<grid_for((size_t)B * H), 256, 0, st>>>(p, o, H, B, w.gout, w.z3, w.d3);
    // Deltas through W3 and W2 (transposed: B(n=i, k=j) = W[j*H + i]) and the weight gradients
    // (sums over samples, ascending; the bias gradients are the same sums of the deltas alone,
    // the row sums of A).  Products that need only deltas already computed share a launch: the
    // delta through W3 with the gradients of W3 and W4, then the delta through W2 with the
    // gradient of W2.
    const OgArgs d2a{B, H, H, w.d3, H, 1, p + o.W3, 1, H, nullptr, w.z2, w.d2, nullptr, H, nullptr};
    const OgArgs gw3{H, H, B, w.d3, 1, H, w.h2, 1, H, nullptr, nullptr, grad + o.W3, nullptr, H, grad + o.b3};
    const OgArgs gw4{1, H, B, w.gout, 0, 1, w.h3, 1, H, nullptr, nullptr, grad + o.W4, nullptr, H, grad + o.b4};
    const OgArgs d1a{B, H, H, w.d2, H, 1, p + o.W2, 1, H, nullptr, w.z1, w.d1, nullptr, H, nullptr};
    const OgArgs gw2{H, H, B, w.d2, 1, H, w.h1, 1, H, nullptr, nullptr, grad + o.W2, nullptr, H, grad + o.b2};
    const dim3 gb = og_grid(B, H), gw = og_grid(H, H);
    const dim3 gz(std::max(gb.x, gw.x), std::max(gb.y, gw.y), 1);
    k_ogemm_bwd<<<dim3(gz.x, gz.y, 3), OG_THREADS, 0, st>>>(d2a, gw3, gw4, 2);
    k_ogemm_bwd<<<dim3(gz.x, gz.y, 2), OG_THREADS, 0, st>>>(d1a, gw2, gw2, 1);
    int JB = 2;   // hidden units per CTA: few, so that the H / JB CTAs reach many SMs
    while (JB > 1 && (JB * N > 1024 || w1grad_smem(JB, D, N) > 48 * 1024)) JB >>= 1;
    if (JB * N <= 1024 && w1grad_smem(JB, D, N) <= 48 * 1024) {
        k_mlp_w1grad<<<(H + JB - 1) / JB, JB * N, w1grad_smem(JB, D, N), st>>>(w.d1, feats, B, N, D, H, JB, grad + o.W1,
                                                                           grad + o.b1);
        count_launch(5);
    } else {
        k_mlp_w1grad_wide<<<grid_for((size_t)H * D, 64), 64, 0, st>>>(w.d1, feats, param_of, B, N, D, H, grad + o.W1);
        k_colsum<<<(H + 127) / 128, 128, 0, st>>>(w.d1, H, B, grad + o.b1);
        count_launch(6);
    }
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

// ------------------------------------------------------------------------------
// surrogate-screened generations
// ------------------------------------------------------------------------------
struct SurrDev {
    unsigned long long n_e;
    int32_t use;         // screen the next generation
    int32_t screened;    // this generation was screened
    float mae, tau;
};

struct SurrogateState {
    ct_surrogate_params cfg{};
    int D = 0;
    MlpOff off{};
    const float* logt = nullptr;
    DevBuf<float> params, mom, grad, work, pred, by;
    DevBuf<int32_t> feats, param_of;
    DevBuf<uint64_t> cand, rep, evk, ek, evk_chosen;
    DevBuf<float> ey;
    DevBuf<uint32_t> in_e;
    DevBuf<SurrDev> sd;
    SurrDev* h_sd = nullptr;   // pinned
    OptDev* h_od = nullptr;    // pinned
    RepairScratch rs;
    size_t e_cap = 0, max_n = 0;
};

void surrogate_free(SurrogateState* g) {
    if (!g) return;
    g->params.release(); g->mom.release(); g->grad.release(); g->work.release(); g->pred.release(); g->by.release();
    g->feats.release(); g->param_of.release(); g->cand.release(); g->rep.release(); g->evk.release(); g->ek.release();
    g->evk_chosen.release(); g->ey.release(); g->in_e.release(); g->sd.release();
    g->rs.release_all();
    if (g->h_sd) cudaFreeHost(g->h_sd);
    if (g->h_od) cudaFreeHost(g->h_od);
    delete g;
}

__global__ void __launch_bounds__(256) k_propose_pool(OptArgs a, uint32_t gen, uint64_t* __restrict__ cand) {
    __shared__ int order[CT_MAX_POP];
    propose_dev(a, gen, cand + (size_t)blockIdx.x * a.P, order, (int)blockIdx.x);
}

__global__ void __launch_bounds__(256) k_post_pool(OptArgs a, uint32_t gen, uint64_t* __restrict__ keys) {
    __shared__ GaMutSmem gm;
    post_repair_dev(a, gen, keys + (size_t)blockIdx.x * a.P, gm, (int)blockIdx.x);
}

__global__ void __launch_bounds__(256) k_select_s(OptArgs a, uint32_t gen, const uint64_t* __restrict__ keys,
                                                  const float* __restrict__ fit) {
    __shared__ SelectSmem sm;
    select_dev(a, gen, keys, fit, sm);
}

// lowest prediction per slot over the pool (ties: smaller key, then smaller pool index)
__global__ void k_surr_choose(int P, int pool, const float* __restrict__ pred, const uint64_t* __restrict__ cand,
                              const uint64_t* __restrict__ rep, const uint64_t* __restrict__ evk,
                              uint64_t* __restrict__ oc, uint64_t* __restrict__ orp, uint64_t* __restrict__ oe) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    int bs = 0;
    float bp = pred[i];
    uint64_t bk = evk[i];
    for (int s = 1; s < pool; ++s) {
        const size_t q = (size_t)s * P + i;
        const float pr = pred[q];
        if (pr < bp || (pr == bp && evk[q] < bk)) { bp = pr; bk = evk[q]; bs = s; }
    }
    const size_t q = (size_t)bs * P + i;
    oc[i] = cand[q];
    orp[i] = rep[q];
    oe[i] = evk[q];
}

// judge (error of the predictions made before learning) and append new evaluations
constexpr int JUDGE_THREADS = 256;

__global__ void __launch_bounds__(JUDGE_THREADS)
k_surr_judge(const uint64_t* __restrict__ keys, int64_t nv, const float* __restrict__ logt,
             const uint64_t* __restrict__ evk, const float* __restrict__ pred, int P, int warm_mult,
             float mae_ratio, int screened, uint32_t* __restrict__ in_e, uint64_t* __restrict__ ek,
             float* __restrict__ ey, SurrDev* sd) {
    __shared__ int64_t rks[CT_MAX_POP];
    __shared__ float ys[CT_MAX_POP], ps[CT_MAX_POP];
    __shared__ uint32_t pos[CT_MAX_POP];
    __shared__ uint32_t wsum[JUDGE_THREADS / 32];
    __shared__ unsigned long long n0_s;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // the rank lookups (binary searches over the valid keys) and whether each configuration is
    // new to the training set, in parallel ...
    for (int i = t; i < P; i += blockDim.x) {
        const int64_t rk = rank_of(keys, nv, evk[i]);
        rks[i] = rk;
        ys[i] = logt[rk];
        ps[i] = pred[i];
    }
    if (t == 0) n0_s = sd->n_e;
    __syncthreads();
    // ... a configuration joins the training set at its first position in this generation, if no
    // earlier generation added it; positions by an exclusive scan over population order
    uint32_t carry = 0;
    for (int c0 = 0; c0 < P; c0 += JUDGE_THREADS) {
        const int i = c0 + t;
        uint32_t fresh = 0;
        if (i < P) {
            const int64_t rk = rks[i];
            fresh = !((in_e[rk >> 5] >> (rk & 31)) & 1u);
            for (int q = 0; q < i && fresh; ++q) fresh = rks[q] != rk;
        }
        uint32_t inc = fresh;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t wb = 0, tot = 0;
        for (int w = 0; w < JUDGE_THREADS / 32; ++w) { wb += w < warp ? wsum[w] : 0u; tot += wsum[w]; }
        if (i < P) pos[i] = fresh ? carry + wb + inc - 1u : ~0u;
        carry += tot;
        __syncthreads();
    }
    for (int i = t; i < P; i += blockDim.x) {
        if (pos[i] == ~0u) continue;
        const size_t n = (size_t)n0_s + pos[i];
        ek[n] = evk[i];
        ey[n] = ys[i];
        atomicOr(in_e + (rks[i] >> 5), 1u << (rks[i] & 31));
    }
    if (t != 0) return;
    // the fp32 sums in ascending i, one thread
    float sa = 0.0f, sy = 0.0f, s_dev = 0.0f;
    for (int i = 0; i < P; ++i) {
        const float y = ys[i];
        sa = __fadd_rn(sa, fabsf(__fsub_rn(ps[i], y)));
        sy = __fadd_rn(sy, y);
    }
    const float mae = __fdiv_rn(sa, (float)P), ybar = __fdiv_rn(sy, (float)P);
    for (int i = 0; i < P; ++i) s_dev = __fadd_rn(s_dev, fabsf(__fsub_rn(ys[i], ybar)));
    const float tau = __fmul_rn(mae_ratio, __fdiv_rn(s_dev, (float)P));
    const unsigned long long n = n0_s + carry;
    sd->n_e = n;
    sd->mae = mae;
    sd->tau = tau;
    sd->screened = screened;
    sd->use = (n >= (unsigned long long)warm_mult * (unsigned long long)P) && mae <= tau;
}

__global__ void k_surr_batch(const DevSpace* __restrict__ sp, const uint64_t* __restrict__ ek,
                             const float* __restrict__ ey, const SurrDev* __restrict__ sd, uint64_t seed, uint32_t gen,
                             uint32_t step, int B, int32_t* __restrict__ feats, float* __restrict__ y) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t n = (uint32_t)sd->n_e;
    const uint32_t pick = uint_below(rng_word(seed, (uint32_t)b, gen, PU_MLP_BATCH, step), n ? n : 1u);
    const uint64_t key = ek[pick];
    int base = 0;
    for (int k = 0; k < sp->n; ++k) {
        feats[(size_t)b * sp->n + k] = base + field(sp, key, k);
        base += sp->r[k];
    }
    y[b] = ey[pick];
}

static ct_status predict_keys(ct_opt* o, const uint64_t* keys, int n, float* out, cudaStream_t st) {
    SurrogateState* g = o->sg;
    k_feats<<<(n + 255) / 256, 256, 0, st>>>(o->s->d, keys, n, g->feats.p);
    count_launch();
    return mlp_forward_impl(g->params.p, g->D, g->cfg.hidden, o->N, g->feats.p, n, out,
                            carve(g->work.p, g->cfg.hidden, (int)g->max_n), st);
}

ct_status surrogate_step(ct_opt* o, uint32_t gen, cudaStream_t st) {
    SurrogateState* g = o->sg;
    ct_space* s = o->s;
    const int P = o->P, pool = g->cfg.pool;
    const bool init = gen == 0 || (o->kind == CT_DE && g->h_od->reinit_pending);
    const bool screened = !init && g->h_sd->use && (gen > 0);
    // the evaluated set can grow by P per generation
    if (g->h_sd->n_e + (uint64_t)P > g->e_cap) {
        const size_t cap = std::max<size_t>(2 * g->e_cap, g->h_sd->n_e + (size_t)P * 64);
        DevBuf<uint64_t> nk;
        DevBuf<float> ny;
        CT_TRY(nk.ensure(cap));
        CT_TRY(ny.ensure(cap));
        if (g->h_sd->n_e) {
            CT_TRY_CUDA(cudaMemcpyAsync(nk.p, g->ek.p, g->h_sd->n_e * 8, cudaMemcpyDeviceToDevice, st));
            CT_TRY_CUDA(cudaMemcpyAsync(ny.p, g->ey.p, g->h_sd->n_e * 4, cudaMemcpyDeviceToDevice, st));
            CT_TRY_CUDA(cudaStreamSynchronize(st));
        }
        g->ek.release();
        g->ey.release();
        g->ek = nk;
        g->ey = ny;
        g->e_cap = cap;
    }
    const OptArgs a = o->args();
    uint64_t* evk = g->evk_chosen.p;
    if (screened) {
        k_propose_pool<<<pool, 256, 0, st>>>(a, gen, g->cand.p);
        count_launch();
        CT_TRY(repair_impl(s, g->rs, g->cand.p, (int64_t)pool * P, g->rep.p, nullptr, st));
        CT_TRY_CUDA(cudaMemcpyAsync(g->evk.p, g->rep.p, (size_t)pool * P * 8, cudaMemcpyDeviceToDevice, st));
        k_post_pool<<<pool, 256, 0, st>>>(a, gen, g->evk.p);
        count_launch();
        CT_TRY(predict_keys(o, g->evk.p, pool * P, g->pred.p, st));
        k_surr_choose<<<(P + 127) / 128, 128, 0, st>>>(P, pool, g->pred.p, g->cand.p, g->rep.p, g->evk.p, o->cand.p,
                                                      o->rep.p, evk);
        count_launch();
    } else {
        k_propose_pool<<<1, 256, 0, st>>>(a, gen, o->cand.p);
        count_launch();
        CT_TRY(repair_impl(s, o->rs, o->cand.p, P, o->rep.p, nullptr, st));
        CT_TRY_CUDA(cudaMemcpyAsync(evk, o->rep.p, (size_t)P * 8, cudaMemcpyDeviceToDevice, st));
        k_post_pool<<<1, 256, 0, st>>>(a, gen, evk);
        count_launch();
    }
    CT_TRY(evaluate_impl(s, o->memo.p, &o->st.p->n_unique, &o->st.p->cost, evk, P, o->fit.p, nullptr, st));
    CT_TRY(predict_keys(o, evk, P, g->pred.p, st));
    k_surr_judge<<<1, JUDGE_THREADS, 0, st>>>(s->keys.p, (int64_t)s->n_valid, g->logt, evk, g->pred.p, P, g->cfg.warmup_mult,
                                   g->cfg.mae_ratio, screened ? 1 : 0, g->in_e.p, g->ek.p, g->ey.p, g->sd.p);
    count_launch();
    const int B = g->cfg.batch, H = g->cfg.hidden;
    for (int t = 0; t < g->cfg.steps; ++t) {
        k_surr_batch<<<(B + 127) / 128, 128, 0, st>>>(s->d, g->ek.p, g->ey.p, g->sd.p, o->seed, gen, (uint32_t)t, B,
                                                      g->feats.p, g->by.p);
        count_launch();
        CT_TRY(mlp_grad_impl(g->params.p, g->D, H, o->N, g->feats.p, g->by.p, B, g->grad.p, g->pred.p + P,
                             g->param_of.p, carve(g->work.p, H, (int)g->max_n), st));
        k_mlp_sgd<<<grid_for(g->off.total), 256, 0, st>>>(g->params.p, g->mom.p, g->grad.p, g->off.total,
                                                          g->cfg.lr, g->cfg.momentum);
        count_launch();
    }
    k_select_s<<<1, 256, 0, st>>>(a, gen, evk, o->fit.p);
    count_launch();
    CT_TRY_CUDA(cudaMemcpyAsync(g->h_sd, g->sd.p, sizeof(SurrDev), cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaMemcpyAsync(g->h_od, o->st.p, sizeof(OptDev), cudaMemcpyDeviceToHost, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

}  // namespace ct

using namespace ct;

extern "C" {

void ct_surrogate_params_default(ct_surrogate_params* p) {
    if (!p) return;
    p->pool = 16; p->hidden = 256; p->batch = 256; p->steps = 8; p->warmup_mult = 4;
    p->lr = 1e-2f; p->momentum = 0.9f; p->mae_ratio = 1.0f;
}

int64_t ct_mlp_param_count(int32_t D, int32_t H) { return (int64_t)mlp_off(D, H).total; }

ct_status ct_mlp_init(int32_t D, int32_t H, uint64_t seed, float* d_params, ct_stream stream) {
    if (D < 1 || H < 1 || !d_params) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    const MlpOff o = mlp_off(D, H);
    const float a1 = sqrtf(6.0f / (float)(D + H)), a2 = sqrtf(6.0f / (float)(H + H)), a4 = sqrtf(6.0f / (float)(H + 1));
    k_mlp_init<<<grid_for(o.total), 256, 0, (cudaStream_t)stream>>>(d_params, o, seed, a1, a2, a2, a4);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

size_t ct_mlp_workspace_bytes(int32_t D, int32_t H, int32_t B) {
    (void)D;
    return work_floats(H, B) * sizeof(float) + (size_t)B * sizeof(float);
}

ct_status ct_mlp_forward(int32_t D, int32_t H, int32_t N, const float* d_params, const int32_t* d_feats, int32_t B,
                         float* d_pred, void* d_work, ct_stream stream) {
    if (D < 1 || H < 1 || N < 1 || B < 1 || !d_params || !d_feats || !d_pred || !d_work) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    return mlp_forward_impl(d_params, D, H, N, d_feats, B, d_pred, carve((float*)d_work, H, B), (cudaStream_t)stream);
}

ct_status ct_mlp_grad(int32_t D, int32_t H, int32_t N, const float* d_params, const int32_t* d_feats,
                      const int32_t* d_param_of, const float* d_y, int32_t B, float* d_grad, void* d_work, ct_stream stream) {
    if (D < 1 || H < 1 || N < 1 || B < 1 || !d_params || !d_feats || !d_param_of || !d_y || !d_grad || !d_work) {
        set_error("bad argument");
        return CT_ERR_INVALID_ARG;
    }
    float* w = (float*)d_work;
    return mlp_grad_impl(d_params, D, H, N, d_feats, d_y, B, d_grad, w + work_floats(H, B), d_param_of,
                         carve(w, H, B), (cudaStream_t)stream);
}

ct_status ct_mlp_sgd(float* d_params, float* d_mom, const float* d_grad, int64_t n, float lr, float mu, ct_stream stream) {
    if (!d_params || !d_mom || !d_grad || n < 0) { set_error("bad argument"); return CT_ERR_INVALID_ARG; }
    k_mlp_sgd<<<grid_for((size_t)n), 256, 0, (cudaStream_t)stream>>>(d_params, d_mom, d_grad, (size_t)n, lr, mu);
    count_launch();
    CT_TRY_CUDA(cudaGetLastError());
    return CT_OK;
}

ct_status ct_opt_set_surrogate(ct_opt* o, const ct_surrogate_params* prm, const float* d_log_table) {
    if (!o || !d_log_table) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    if (o->kind != CT_DE && o->kind != CT_GA) { set_error("the surrogate screens DE and GA runs only"); return CT_ERR_INVALID_ARG; }
    if (o->sg) { set_error("surrogate already set"); return CT_ERR_STATE; }
    if (o->prm.repair_rule || !o->prm.constraint_aware) {
        set_error("surrogate screening runs on the constraint-aware method with the Hamming repair");
        return CT_ERR_INVALID_ARG;
    }
    ct_surrogate_params cfg;
    if (prm) cfg = *prm; else ct_surrogate_params_default(&cfg);
    if (cfg.pool < 1 || cfg.pool > 64 || cfg.hidden < 1 || cfg.hidden > 1024 || cfg.batch < 1 || cfg.batch > 4096 ||
        cfg.steps < 0 || cfg.warmup_mult < 0) {
        set_error("surrogate parameters out of range");
        return CT_ERR_INVALID_ARG;
    }
    SurrogateState* g = new (std::nothrow) SurrogateState();
    if (!g) { set_error("host allocation failed"); return CT_ERR_OOM; }
    g->cfg = cfg;
    g->logt = d_log_table;
    const ct_space* s = o->s;
    g->D = 0;
    std::vector<int32_t> pof;
    for (int k = 0; k < s->h.n; ++k) { for (int v = 0; v < s->h.r[k]; ++v) pof.push_back(k); g->D += s->h.r[k]; }
    g->off = mlp_off(g->D, cfg.hidden);
    const int P = o->P;
    g->max_n = std::max<size_t>((size_t)cfg.pool * P, (size_t)cfg.batch);
    ct_status e = CT_OK;
#define ALLOC(b, n) if (e == CT_OK) e = g->b.ensure(n)
    ALLOC(params, g->off.total); ALLOC(mom, g->off.total); ALLOC(grad, g->off.total);
    ALLOC(work, work_floats(cfg.hidden, (int)g->max_n)); ALLOC(pred, g->max_n + cfg.batch); ALLOC(by, std::max(cfg.batch, P));
    ALLOC(feats, g->max_n * s->h.n); ALLOC(param_of, pof.size()); ALLOC(cand, (size_t)cfg.pool * P);
    ALLOC(rep, (size_t)cfg.pool * P); ALLOC(evk, (size_t)cfg.pool * P); ALLOC(evk_chosen, P);
    ALLOC(in_e, (s->n_valid + 31) / 32); ALLOC(sd, 1);
#undef ALLOC
    if (e == CT_OK) e = repair_reserve(g->rs, (int64_t)cfg.pool * P);
    if (e == CT_OK && (cudaMallocHost(&g->h_sd, sizeof(SurrDev)) != cudaSuccess ||
                       cudaMallocHost(&g->h_od, sizeof(OptDev)) != cudaSuccess)) {
        set_error("pinned allocation failed");
        e = CT_ERR_OOM;
    }
    if (e == CT_OK) {
        memset(g->h_sd, 0, sizeof(SurrDev));
        memset(g->h_od, 0, sizeof(OptDev));
        if (cudaMemcpy(g->param_of.p, pof.data(), pof.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(g->mom.p, 0, g->off.total * 4) != cudaSuccess ||
            cudaMemset(g->in_e.p, 0, ((s->n_valid + 31) / 32) * 4) != cudaSuccess ||
            cudaMemset(g->sd.p, 0, sizeof(SurrDev)) != cudaSuccess) {
            set_error("initialising the surrogate failed");
            e = CT_ERR_CUDA;
        }
    }
    if (e == CT_OK) e = ct_mlp_init(g->D, cfg.hidden, o->seed, g->params.p, nullptr);
    if (e == CT_OK && cudaDeviceSynchronize() != cudaSuccess) { set_error("surrogate init failed"); e = CT_ERR_CUDA; }
    if (e != CT_OK) { surrogate_free(g); return e; }
    o->sg = g;
    return CT_OK;
}

ct_status ct_opt_surrogate_info(ct_opt* o, int32_t* screened, int32_t* use_next, float* mae, float* tau,
                                uint64_t* n_evaluated, float* d_params, ct_stream stream) {
    if (!o || !o->sg) { set_error("run has no surrogate"); return CT_ERR_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    SurrDev h;
    CT_TRY_CUDA(cudaMemcpyAsync(&h, o->sg->sd.p, sizeof h, cudaMemcpyDeviceToHost, st));
    if (d_params)
        CT_TRY_CUDA(cudaMemcpyAsync(d_params, o->sg->params.p, o->sg->off.total * 4, cudaMemcpyDeviceToDevice, st));
    CT_TRY_CUDA(cudaStreamSynchronize(st));
    if (screened) *screened = h.screened;
    if (use_next) *use_next = h.use;
    if (mae) *mae = h.mae;
    if (tau) *tau = h.tau;
    if (n_evaluated) *n_evaluated = h.n_e;
    return CT_OK;
}

ct_status ct_opt_last_generation(const ct_opt* o, uint64_t* d_cand, uint64_t* d_rep, uint64_t* d_eval, float* d_fit,
                                 ct_stream stream) {
    if (!o) { set_error("null argument"); return CT_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    CT_TRY(o->wait_ready(st));
    const size_t P = o->P;
    const uint64_t* ev = o->sg ? o->sg->evk_chosen.p : o->rep.p;
    if (d_cand) CT_TRY_CUDA(cudaMemcpyAsync(d_cand, o->cand.p, P * 8, cudaMemcpyDeviceToDevice, st));
    if (d_rep) CT_TRY_CUDA(cudaMemcpyAsync(d_rep, o->rep.p, P * 8, cudaMemcpyDeviceToDevice, st));
    if (d_eval) CT_TRY_CUDA(cudaMemcpyAsync(d_eval, ev, P * 8, cudaMemcpyDeviceToDevice, st));
    if (d_fit) CT_TRY_CUDA(cudaMemcpyAsync(d_fit, o->fit.p, P * 4, cudaMemcpyDeviceToDevice, st));
    return CT_OK;
}

}  // extern "C"
