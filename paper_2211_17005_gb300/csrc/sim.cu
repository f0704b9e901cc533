// Inner-default kernel of the hierarchical CVA simulation, and the dispatch
// of the outer-path kernel instantiations (outer_*.cu).
//
// Inner defaults (Sec. 3.2 / eq. (e:tau)), two kernels:
//   inner_count_kernel   one warp per outer path: N default clocks per
//     counterparty; tau^{k,l} falls in (t_{j-1}, t_j] when the uniform w
//     (epsilon = -log(1 - w)) satisfies T(j-1) < w <= T(j), T = 1 - e^{-Lambda};
//     the default step is the lower bound of w in the monotone thresholds, and
//     the integer count of defaults per (counterparty, step) goes to global memory;
//   inner_target_kernel  one thread per outer path: the averaged target of eq.
//     (eq:CVA_portfolio) of every portfolio from the counts,
//       xi_bar_i = beta_i^{-1} (1/N) sum_{j>i} sum_c V_c(j) count_c(j),
//     as a running sum over the dates from the last, every load and store
//     coalesced over consecutive paths.
// The counts are integers, so the targets do not depend on the order of the draws.
#include <mutex>

#include "cva_internal.h"
#include "rng.cuh"

namespace cva {

namespace {

struct InnerArgs {
    uint32_t M, k0, seed_lo, seed_hi, N;
    uint32_t branch;                  // third counter word of the clocks (twin copy id, 0 otherwise)
    int n, NPF, P;
    const float *__restrict__ thr;    // [n+1][C][M]
    const float *__restrict__ expo;   // [NPF][n+1][C][M]
    const float *__restrict__ disc;   // [n+1][M]
    float *targets;                   // [NPF][n][M]
    uint8_t *idx;                     // [M][N][C] or null
    uint16_t *cnt16;                  // [n+1][C][M] default counts (N <= 65535) ...
    uint32_t *cnt32;                  // ... or these (larger N)
};

// First j in [1, n] with T(j) >= w for nondecreasing thresholds T, else n + 1
// (n <= 255): the lower bound by the fixed power-of-two steps 128, 64, ..., 1 (every
// lane of a warp runs the same unrolled steps, so that the searches of several
// counterparties interleave; a step past n reads nothing).
template <class Thr>
__device__ __forceinline__ int lower_bound_pow2(Thr T, int n, float w)
{
    int pos = 0;   // T(1..pos) < w
#pragma unroll
    for (int step = 128; step > 0; step >>= 1) {
        const int q = pos + step;
        if (q <= n && T(q) < w) pos = q;
    }
    return pos + 1;
}

template <int C>
__global__ void __launch_bounds__(256) inner_count_kernel(InnerArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int P = a.P, n = a.n, np1 = n + 1;
    float *thr_s = reinterpret_cast<float *>(smem);                 // [P][C][n+1]
    // counters [P][C][n+1]: two 16-bit counters per word when every count fits (N <= 65535)
    uint32_t *cnt_s = reinterpret_cast<uint32_t *>(thr_s + P * C * np1);
    const bool packed = a.cnt16 != nullptr;
    const int n_words = packed ? (P * C * np1 + 1) / 2 : P * C * np1;
    const uint32_t M = a.M, tile0 = blockIdx.x * (uint32_t)P;
    const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = nthr >> 5;

    for (int i = tid; i < n * C * P; i += nthr) {
        const int pk = i % P, jc = i / P, c = jc % C, j = 1 + jc / C;
        const uint32_t kl = tile0 + pk;
        thr_s[(pk * C + c) * np1 + j] = (kl < M) ? __ldg(a.thr + ((size_t)j * C + c) * M + kl) : 2.f;
    }
    for (int i = tid; i < n_words; i += nthr) cnt_s[i] = 0u;
    __syncthreads();

    for (int pk = warp; pk < P; pk += nwarps) {
        const uint32_t kl = tile0 + pk;
        if (kl >= M) continue;
        const uint32_t k = a.k0 + kl;
        for (uint32_t l = lane; l < a.N; l += 32) {
#pragma unroll
            for (int cb = 0; cb < (C + 3) / 4; ++cb) {
                const uint4 x = philox4x32_10(make_uint4(k, l, a.branch, (kStreamInner << 24) | (uint32_t)cb),
                                              a.seed_lo, a.seed_hi);
                const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * cb + i;
                    if (c < C) {
                        const float w = uniform23(xs[i]);
                        const float *T = thr_s + (pk * C + c) * np1;
                        const int lo = lower_bound_pow2([T](int j) { return T[j]; }, n, w);
                        if (a.idx) a.idx[((size_t)kl * a.N + l) * C + c] = (uint8_t)lo;
                        if (lo <= n) {
                            const int ci = (pk * C + c) * np1 + lo;
                            if (packed) atomicAdd(&cnt_s[ci >> 1], 1u << (16 * (ci & 1)));
                            else atomicAdd(&cnt_s[ci], 1u);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    // the counts of steps 1..n, P consecutive paths per (step, counterparty) row
    for (int i = tid; i < n * C * P; i += nthr) {
        const int pk = i % P, jc = i / P, c = jc % C, j = 1 + jc / C;
        const uint32_t kl = tile0 + pk;
        if (kl < M) {
            const int ci = (pk * C + c) * np1 + j;
            const uint32_t v = packed ? (cnt_s[ci >> 1] >> (16 * (ci & 1))) & 0xffffu : cnt_s[ci];
            const size_t o = ((size_t)j * C + c) * M + kl;
            if (a.cnt16) a.cnt16[o] = (uint16_t)v;
            else a.cnt32[o] = v;
        }
    }
}

template <int C>
__global__ void __launch_bounds__(256) inner_target_kernel(InnerArgs a)
{
    const uint32_t kl = blockIdx.x * blockDim.x + threadIdx.x;
    if (kl >= a.M) return;
    const size_t M = a.M;
    const int n = a.n, np1 = n + 1, NPF = a.NPF;
    const float invN = 1.0f / (float)a.N;
    float S[kMaxPF];   // sum_{j > i} sum_c V_c(j) count_c(j) of each portfolio
#pragma unroll
    for (int pf = 0; pf < kMaxPF; ++pf) S[pf] = 0.f;
    for (int j = n; j >= 1; --j) {
        float cnt[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const size_t o = ((size_t)j * C + c) * M + kl;
            cnt[c] = a.cnt16 ? (float)__ldg(a.cnt16 + o) : (float)__ldg(a.cnt32 + o);
        }
        const float bi = expf(__ldg(a.disc + (size_t)(j - 1) * M + kl)) * invN;   // beta_{j-1}^{-1} / N
#pragma unroll
        for (int pf = 0; pf < kMaxPF; ++pf) {
            if (pf < NPF) {
                float h = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c)
                    h = fmaf(__ldg(a.expo + ((size_t)(pf * np1 + j) * C + c) * M + kl), cnt[c], h);
                S[pf] += h;
                a.targets[((size_t)pf * n + j - 1) * M + kl] = S[pf] * bi;
            }
        }
    }
}

// Sampling statistics of Prop. 1 (Sec. ss:choice1). For the pointwise loss
// g_l = (xi^{k,l}_i - phi_i(Y^k))^2 of the first two inner draws l = 0, 1 of path
// k (single-draw targets of eq. (eq:CVA_portfolio): the same clocks as the
// simulation's draws 0 and 1), block sums over paths, per date i in [1, n-1], of
// (g0 + g1)/2, (g0^2 + g1^2)/2 and g0 g1, in FP64: part[block][n][3] (date 0 zero).
struct OversimArgs {
    uint32_t M, k0, seed_lo, seed_hi;
    int n, pf;
    const float *__restrict__ thr;    // [n+1][C][M]
    const float *__restrict__ expo;   // [NPF][n+1][C][M]
    const float *__restrict__ disc;   // [n+1][M]
    const float *__restrict__ pred;   // [n][M]
    double *part;
};

template <int C>
__global__ void __launch_bounds__(256) oversim_kernel(OversimArgs a)
{
    __shared__ double red[8][3];
    const uint32_t M = a.M, kl = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = kl < M;
    const int n = a.n, np1 = n + 1, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int idx[2][C];
    float vs[2][C];
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            idx[l][c] = n + 1;
            vs[l][c] = 0.f;
        }
    if (live) {
        const uint32_t k = a.k0 + kl;
#pragma unroll
        for (int l = 0; l < 2; ++l)
#pragma unroll
            for (int cb = 0; cb < (C + 3) / 4; ++cb) {
                const uint4 x = philox4x32_10(make_uint4(k, (uint32_t)l, 0u, (kStreamInner << 24) | (uint32_t)cb),
                                              a.seed_lo, a.seed_hi);
                const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = 4 * cb + t;
                    if (c < C) {
                        const float w = uniform23(xs[t]);
                        const float *Tc = a.thr + (size_t)c * M + kl;   // T(j) at Tc[j C M]
                        const int lo = lower_bound_pow2([Tc, M](int j) { return __ldg(Tc + (size_t)j * C * M); },
                                                        n, w);
                        idx[l][c] = lo;
                        if (lo <= n) vs[l][c] = __ldg(a.expo + ((size_t)(a.pf * np1 + lo) * C + c) * M + kl);
                    }
                }
            }
    }
    for (int i = 1; i < n; ++i) {
        double s[3] = {0.0, 0.0, 0.0};
        if (live) {
            float h0 = 0.f, h1 = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (idx[0][c] > i) h0 += vs[0][c];
                if (idx[1][c] > i) h1 += vs[1][c];
            }
            const float e = expf(__ldg(a.disc + (size_t)i * M + kl));
            const double f = (double)__ldg(a.pred + (size_t)i * M + kl);
            const double g0 = ((double)(h0 * e) - f) * ((double)(h0 * e) - f),
                         g1 = ((double)(h1 * e) - f) * ((double)(h1 * e) - f);
            s[0] = 0.5 * (g0 + g1);
            s[1] = 0.5 * (g0 * g0 + g1 * g1);
            s[2] = g0 * g1;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
            if (lane == 0) red[warp][q] = s[q];
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
            a.part[((size_t)blockIdx.x * n + i) * 3 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) a.part[(size_t)blockIdx.x * n * 3 + threadIdx.x] = 0.0;
}

}  // namespace

cva_status launch_oversim(const Sim &s, int pf, const float *pred, uint64_t seed, double *part, unsigned blocks,
                          cudaStream_t st)
{
    OversimArgs a;
    a.M = (uint32_t)s.M;
    a.k0 = 0;
    a.seed_lo = (uint32_t)seed;
    a.seed_hi = (uint32_t)(seed >> 32);
    a.n = s.n;
    a.pf = pf;
    a.thr = s.d_thr;
    a.expo = s.d_expo;
    a.disc = s.d_disc;
    a.pred = pred;
    a.part = part;
    static constexpr void (*by_c[kMaxC])(OversimArgs) = {
        oversim_kernel<1>,  oversim_kernel<2>,  oversim_kernel<3>,  oversim_kernel<4>,
        oversim_kernel<5>,  oversim_kernel<6>,  oversim_kernel<7>,  oversim_kernel<8>,
        oversim_kernel<9>,  oversim_kernel<10>, oversim_kernel<11>, oversim_kernel<12>,
        oversim_kernel<13>, oversim_kernel<14>, oversim_kernel<15>, oversim_kernel<16>};
    if (s.C < 1 || s.C > kMaxC) return fail(CVA_ENOTSUP, "oversimulation statistics: 1 <= C <= 16");
    by_c[s.C - 1]<<<blocks, 256, 0, st>>>(a);
    CVA_CUDA_TRY(cudaGetLastError());
    return CVA_OK;
}

// Registry of the compiled outer-kernel shapes (one translation unit each).
int outer_insts_small(const OuterInst **out);
int outer_insts_paper(const OuterInst **out);
int outer_insts_batched(const OuterInst **out);
int outer_insts_generic(const OuterInst **out);

static const OuterInst *find_outer(int E, int C, int CS, int G, int NPF)
{
    const OuterInst *best = nullptr;
    int (*tables[])(const OuterInst **) = {outer_insts_small, outer_insts_paper, outer_insts_batched};
    for (auto tab : tables) {
        const OuterInst *p = nullptr;
        const int cnt = tab(&p);
        for (int i = 0; i < cnt; ++i) {
            const OuterInst &o = p[i];
            if (o.E == E && o.C == C && o.CS == CS && o.NPF == NPF && o.G >= G && (!best || o.G < best->G))
                best = &o;
        }
    }
    return best;
}

bool outer_supported(int E, int C, int CS, int G, int NPF, int *Ginst)
{
    const OuterInst *o = find_outer(E, C, CS, G, NPF);
    if (o && Ginst) *Ginst = o->G;
    return o != nullptr;
}

void forget_const_owner(const Sim *s)
{
    int (*tables[])(const OuterInst **) = {outer_insts_small, outer_insts_paper, outer_insts_batched,
                                           outer_insts_generic};
    for (auto tab : tables) {
        const OuterInst *p = nullptr;
        const int cnt = tab(&p);
        for (int i = 0; i < cnt; ++i) p[i].forget(s);
    }
}

static const OuterInst *generic_outer()
{
    const OuterInst *p = nullptr;
    outer_insts_generic(&p);
    return p;
}

cva_status launch_adjoint(Sim &s, const AdjBuffers &b, uint64_t seed, uint64_t k0, uint32_t M, cudaStream_t st)
{
    if (s.generic) return generic_outer()->adjoint(s, b, seed, k0, M, st);
    const OuterInst *o = find_outer(s.E, s.C, s.CS, s.G, s.NPF);
    if (!o || o->G != s.Ginst || !o->adjoint) return fail(CVA_ENOTSUP, "no adjoint kernel for this model shape");
    return o->adjoint(s, b, seed, k0, M, st);
}

cva_status launch_outer(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    if (s.generic) return generic_outer()->launch(s, seed, k0, st);
    const OuterInst *o = find_outer(s.E, s.C, s.CS, s.G, s.NPF);
    if (!o || o->G != s.Ginst) return fail(CVA_ENOTSUP, "no outer kernel for this model shape");
    return o->launch(s, seed, k0, st);
}

// thresholds (FP32) and counters (16-bit pairs when packed) of P paths
static size_t inner_smem(int P, int C, int n, bool packed)
{
    const size_t cells = (size_t)P * C * (n + 1);
    return 4 * cells + 4 * (packed ? (cells + 1) / 2 : cells);
}

template <int C>
static cudaError_t launch_inner_t(const InnerArgs &args, size_t smem, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(inner_count_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned blocks = (args.M + args.P - 1) / args.P;
    inner_count_kernel<C><<<blocks, 32 * args.P, smem, st>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    inner_target_kernel<C><<<(args.M + 255) / 256, 256, 0, st>>>(args);
    return cudaGetLastError();
}

cva_status launch_inner(Sim &s, uint64_t seed, uint64_t k0, cudaStream_t st)
{
    InnerArgs args;
    args.M = (uint32_t)s.M;
    args.k0 = (uint32_t)k0;
    args.seed_lo = (uint32_t)seed;
    args.seed_hi = (uint32_t)(seed >> 32);
    args.N = s.N;
    args.branch = s.branch;
    args.n = s.n;
    args.NPF = s.NPF;
    int P = (s.tune_inner_P >= 1 && s.tune_inner_P <= 8) ? s.tune_inner_P : 8;
    const bool packed = s.N <= 65535u;
    while (P > 1 && inner_smem(P, s.C, s.n, packed) > 160 * 1024) P >>= 1;
    args.P = P;
    args.thr = s.d_thr;
    args.expo = s.d_expo;
    args.disc = s.d_disc;
    args.targets = s.d_targets;
    args.idx = s.d_idx;
    args.cnt16 = packed ? static_cast<uint16_t *>(s.d_cnt) : nullptr;
    args.cnt32 = packed ? nullptr : static_cast<uint32_t *>(s.d_cnt);
    const size_t smem = inner_smem(P, s.C, s.n, packed);
    static constexpr cudaError_t (*by_c[kMaxC])(const InnerArgs &, size_t, cudaStream_t) = {
        launch_inner_t<1>,  launch_inner_t<2>,  launch_inner_t<3>,  launch_inner_t<4>,
        launch_inner_t<5>,  launch_inner_t<6>,  launch_inner_t<7>,  launch_inner_t<8>,
        launch_inner_t<9>,  launch_inner_t<10>, launch_inner_t<11>, launch_inner_t<12>,
        launch_inner_t<13>, launch_inner_t<14>, launch_inner_t<15>, launch_inner_t<16>};
    if (s.C < 1 || s.C > kMaxC) return fail(CVA_ENOTSUP, "inner kernel: 1 <= C <= 16");
    const cudaError_t e = by_c[s.C - 1](args, smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "inner kernels launch");
    return CVA_OK;
}

}  // namespace cva
