// Pricing of every portfolio on the tensor cores (included by outer.cuh, inside its
// anonymous namespace; uses its constant tables and OuterArgs).
//
// For a pricing date, the date-bucketed MtM of App. B regrouped by (counterparty,
// currency, reset date) is a contraction over (economy e, reset date g):
//   MtM_{pf,c} = sum_e sum_g ( chi_e D_e[g] wA[pf][c][e][g] - chi_e Z_e[g] wK[pf][c][e][g] ),
// the path's bond-price differences D and bond prices Z (times the FX rate chi) against
// the weights, which do not depend on the path or the date. With X the paths' rows
// [chi_e D_e | chi_e Z_e] (K = E x 2G, padded to multiples of 8 per economy) and W the
// weights [NPF C][K], the MtM of 128 paths is the 128 x (NPF C) product X W^T.
//
// The product runs on tcgen05 in TF32 with the FP32 accuracy of the CUDA-core form
// recovered by splitting each operand into a TF32 head and a TF32 tail (x = hi + lo,
// lo = tf32(x - hi), 21 significant bits): X W^T ~ Xhi Whi^T + Xhi Wlo^T + Xlo Whi^T,
// three MMAs per K step accumulating in FP32 in tensor memory (the dropped Xlo Wlo^T
// term is below 2^-22 of each product). The CUDA cores compute the bond prices of
// their path (one thread per path, the chained expm1 differences of price_kernel) and
// write the X row of one economy at a time into one of two shared-memory buffers,
// while the tensor core multiplies the previous economy's.
//
// Persistent blocks of four independent slots of 128 threads (16 warps, so that the
// bond-price chains of one slot hide the latencies of the others): slot s of block b
// takes the work items (path tile t of 128 paths, date j) i = 4 b + s, 4 b + s +
// 4 gridDim.x, ... with j = i / tiles, t = i % tiles. The weights (both TF32 parts)
// are staged once per block; each slot has its own X buffer, accumulator and mbarrier,
// and computes the next economy's bond prices while the tensor core multiplies the
// current one.
//
// Shared memory: W hi | W lo ([NN][KT] each, K-major core matrices), then one X
// buffer per slot, Xhi | Xlo ([128][GK] each). TMEM: a 128 x NN FP32 accumulator per
// slot.
constexpr uint32_t kPriceMbarPolls = 1u << 26;   // limit of a wait for the tensor core
constexpr int kPriceSlots = 4;

template <int E, int G, int NPF, int C>
struct PriceTc {
    static constexpr int GK = (2 * G + 7) / 8 * 8;       // K of one economy: G differences, G prices, padding
    static constexpr int KT = E * GK;                     // K of the whole product
    static constexpr int NN = (NPF * C + 15) / 16 * 16;   // N: every (portfolio, counterparty), padded
    static constexpr uint32_t slot_cols = NN <= 32 ? 32u : NN <= 64 ? 64u : NN <= 128 ? 128u : 256u;
    static constexpr uint32_t tmem_cols = kPriceSlots * slot_cols;
    static constexpr int sWhi = 0, sWlo = NN * KT * 4;
    static constexpr int sX = 2 * NN * KT * 4;            // slot s: Xhi at sX + s xbuf, Xlo at + 128 GK 4
    static constexpr int xbuf = 2 * 128 * GK * 4;
    static constexpr int bytes = sX + kPriceSlots * xbuf;
    static_assert(tmem_cols <= 512, "tensor memory");
    static_assert(bytes <= 220 * 1024, "shared memory");
};

// one answer per slot (its 128 threads, named barrier 1 + slot)
__device__ __forceinline__ bool slot_all(bool p, int slot)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(1 + slot)
        : "memory");
    return r != 0;
}

// the bond prices of one economy for one path (price_kernel's chain), times the FX
// rate: x = [chi D | chi Z | 0]
template <int G, int GK>
__device__ __forceinline__ void price_row(float (&x)[GK], const float4 *tab, int p, float re, float fixm1, float chi)
{
    const float4 tp = __ldg(tab + (p < G ? p : G - 1));   // p >= G: every swap has matured
    const float z_first = expf(fmaf(-tp.y, re, tp.x));
    float zp = 0.f;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        float Z, D;
        if (g < p) {
            Z = 0.f;
            D = 0.f;
        } else if (g == p) {
            Z = z_first;
            D = z_first * fixm1;
        } else {
            const float4 t4 = __ldg(tab + g);
            const float em = expm1_small(fmaf(-t4.w, re, t4.z));
            D = -zp * em;
            Z = fmaf(zp, em, zp);
        }
        zp = Z;
        x[g] = chi * D;
        x[G + g] = chi * Z;
    }
#pragma unroll
    for (int g = 2 * G; g < GK; ++g) x[g] = 0.f;
}

template <int E, int C, int CS, int G, int NPF>
__global__ void __launch_bounds__(128 * kPriceSlots, 1) price_tc_kernel(OuterArgs a, uint32_t tiles)
{
    using P = PriceTc<E, G, NPF, C>;
    constexpr int F = 2 * E - 1 + CS, GK = P::GK, KT = P::KT, NN = P::NN;
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[kPriceSlots];
    const int tid = threadIdx.x, warp = tid >> 5, slot = tid >> 7, row = tid & 127;

    if (warp == 0) {
        umma::tmem_alloc(&s_tmem, P::tmem_cols);
        umma::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < kPriceSlots; ++q) umma::mbar_init(&s_mbar[q], 1);
        umma::fence_mbar_init();
    }
    // the weights as TF32 head and tail: row n = pf C + c, column e GK + g: wA (g < G),
    // then -wK (G <= g < 2G), then zeros
    for (int i = tid; i < NN * KT; i += blockDim.x) {
        const int n = i / KT, k = i % KT, e = k / GK, g = k % GK;
        float w = 0.f;
        if (n < NPF * C && g < 2 * G) {
            const int pf = n / C, c = n % C, wrow = (pf * C + c) * E + e;
            w = g < G ? __ldg(a.w_glob + wrow * G + g) : -__ldg(a.w_glob + kMaxW + wrow * G + (g - G));
        }
        const float hi = umma::tf32_round(w);
        const uint32_t off = umma::kmajor_offset32((uint32_t)n, (uint32_t)k, KT);
        *reinterpret_cast<float *>(tsm + P::sWhi + off) = hi;
        *reinterpret_cast<float *>(tsm + P::sWlo + off) = umma::tf32_round(w - hi);
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = s_tmem + (uint32_t)slot * P::slot_cols;
    const uint32_t sbase = umma::smem_u32(tsm);
    const uint32_t idesc = umma::idesc_tf32_f32(128u, (uint32_t)NN);
    unsigned char *xh = tsm + P::sX + slot * P::xbuf, *xl = xh + 128 * GK * 4;
    const uint32_t ah = sbase + P::sX + (uint32_t)slot * P::xbuf, al = ah + 128u * GK * 4u;
    uint64_t *mbar = &s_mbar[slot];

    const size_t M = a.M;
    const int n = c_sim.n, ppp = c_sim.ppp;
    uint32_t ph = 0;
    bool ok = true;
    const uint32_t items = tiles * (uint32_t)(n + 1);
    for (uint32_t it = blockIdx.x * kPriceSlots + slot; it < items && ok; it += gridDim.x * kPriceSlots) {
        const int j = (int)(it / tiles);
        const uint32_t kl = (it % tiles) * 128u + (uint32_t)row;
        const bool live = kl < a.M;
        const uint32_t kr = live ? kl : 0u;      // a valid path to read for a row past M
        if (j == 0) {   // no default at t_0: exposures of date 0 are never used
            if (live)
                for (int q = 0; q < NPF * C; ++q) {
                    const size_t o = ((size_t)((q / C) * (n + 1)) * C + q % C) * M + kl;
                    a.expo[o] = 0.f;
                    if (a.mtm) a.mtm[o] = 0.f;
                }
            continue;
        }
        const int p = __ldg(a.date_p + j);          // t_j in (p delta, (p+1) delta]
        const float2 *fx = a.fix + (size_t)p * E;
        const float *fe = a.features + (size_t)j * F * M + kr;
        const float *ffix = a.features + (size_t)(p * ppp) * F * M + kr;   // state at the last reset
        const float beta = expf(-__ldg(a.disc + (size_t)j * M + kr));
        float x[GK];
        // the state of economy 1 is requested before economy 0's bond prices are computed,
        // and every later economy's one economy ahead (rates, FX log-level, rate at the fixing)
        float n_r = 0.f, n_fix = 0.f, n_lchi = 0.f;
        if (E > 1) {
            n_r = __ldg(fe + M);
            n_fix = __ldg(ffix + M);
            n_lchi = __ldg(fe + (size_t)E * M);
        }
        {
            const float2 f2 = __ldg(fx);
            price_row<G, GK>(x, a.zc + (size_t)j * E * G, p, __ldg(fe), expm1f(fmaf(f2.y, __ldg(ffix), -f2.x)), 1.f);
        }
        for (int e = 0; e < E; ++e) {
#pragma unroll
            for (int q = 0; q < GK / 4; ++q) {
                float4 h, l;
                h.x = umma::tf32_round(x[4 * q + 0]);
                h.y = umma::tf32_round(x[4 * q + 1]);
                h.z = umma::tf32_round(x[4 * q + 2]);
                h.w = umma::tf32_round(x[4 * q + 3]);
                l.x = umma::tf32_round(x[4 * q + 0] - h.x);
                l.y = umma::tf32_round(x[4 * q + 1] - h.y);
                l.z = umma::tf32_round(x[4 * q + 2] - h.z);
                l.w = umma::tf32_round(x[4 * q + 3] - h.w);
                const uint32_t off = umma::kmajor_offset32((uint32_t)row, (uint32_t)(4 * q), GK);
                *reinterpret_cast<float4 *>(xh + off) = h;
                *reinterpret_cast<float4 *>(xl + off) = l;
            }
            umma::fence_proxy_async();
            umma::fence_before_sync();
            asm volatile("bar.sync %0, 128;" ::"r"(1 + slot) : "memory");
            umma::fence_after_sync();
            if (row == 0) {
                const uint32_t asbo = (GK / 4) * 128u, bsbo = (KT / 4) * 128u;
#pragma unroll
                for (int s = 0; s < GK / 8; ++s) {
                    const uint32_t bk = (uint32_t)((e * GK + 8 * s) / 4) * 128u;
                    const uint64_t dah = umma::smem_desc(ah + s * 256u, 128u, asbo),
                                   dal = umma::smem_desc(al + s * 256u, 128u, asbo),
                                   dbh = umma::smem_desc(sbase + P::sWhi + bk, 128u, bsbo),
                                   dbl = umma::smem_desc(sbase + P::sWlo + bk, 128u, bsbo);
                    umma::mma_tf32(tmem, dah, dbh, idesc, (e > 0 || s > 0) ? 1u : 0u);
                    umma::mma_tf32(tmem, dah, dbl, idesc, 1u);
                    umma::mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
                umma::commit(mbar);
            }
            if (e + 1 < E) {   // the next economy's bond prices while the tensor core works
                const float re = n_r, rfix = n_fix, lchi = n_lchi;   // economy e + 1, requested earlier
                if (e + 2 < E) {
                    n_r = __ldg(fe + (size_t)(e + 2) * M);
                    n_fix = __ldg(ffix + (size_t)(e + 2) * M);
                    n_lchi = __ldg(fe + (size_t)(E + e + 1) * M);   // log chi^{e+2}
                }
                const float2 f2 = __ldg(fx + e + 1);
                const float fixm1 = expm1f(fmaf(f2.y, rfix, -f2.x));
                const float chi = expf(lchi);   // chi^{e+1} from log chi^{e+1}
                price_row<G, GK>(x, a.zc + ((size_t)j * E + e + 1) * G, p, re, fixm1, chi);
            }
            const bool done = umma::mbar_wait(mbar, ph, kPriceMbarPolls);
            ph ^= 1u;
            umma::fence_after_sync();
            ok = slot_all(done && ok, slot);
            if (!ok) break;
        }
        // epilogue: this thread's row of the accumulator, exposures of every (pf, c)
        float mt[NN];
#pragma unroll
        for (int c0 = 0; c0 < NN; c0 += 16) {
            float v[16];
            umma::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0, v);
            umma::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) mt[c0 + i] = v[i];
        }
        if (live)
#pragma unroll
            for (int q = 0; q < NPF * C; ++q) {
                const int pf = q / C, c = q % C;
                const size_t o = ((size_t)(pf * (n + 1) + j) * C + c) * M + kl;
                const float m = ok ? mt[q] : __int_as_float(0x7fc00000);   // a wait that gave up: NaN
                a.expo[o] = c_sim.lgd[c] * beta * fmaxf(m, 0.f);
                if (a.mtm) a.mtm[o] = m;
            }
        // the slot has read its accumulator before its next item's first MMA resets it
        umma::fence_before_sync();
        asm volatile("bar.sync %0, 128;" ::"r"(1 + slot) : "memory");
        umma::fence_after_sync();
    }
    // after a wait that gave up, the slot's MMAs still in flight complete (bounded)
    // before the accumulators are freed
    if (!ok) (void)umma::mbar_wait(mbar, ph, kPriceMbarPolls);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(s_tmem, P::tmem_cols);
}
