// Michelson TDI 1.5 / 2.0 (Sec. II B, Eqs. X1.5, X2.0), mixed precision,
// frozen delays, link and output series on one sample grid: per-link combined
// filters.
//
// Each TDI term is one link series delayed by a sum of light times taken at
// the output time (the frozen form).  Over 512 consecutive output samples the
// fractional part of such a delay moves by at most a few 1e-5 samples (the
// light times change at |dL/dt|/c ~ 3e-8), so the term's 32 Lagrange weights
// at block offset di are, to first order,
//   w_p(f + a di) = w_p(f) + a di w'_p(f),
// with a remainder (a di)^2/2 sum_p |w''_p| < 4.3 (a di)^2 of the largest link
// value (sum_p |w''_p| < 8.5 for eps in [-0.01, 1.01]); with |a di| <= 1e-4
// that is below 5e-8.  All terms that delay the same link then add up to one
// filter of (spread of their delays + 32) taps with a value and a drift
// coefficient per tap for each of the two channels the link enters (X: links
// 2..5, Y: 0, 1, 4, 5, Z: 0..3):
//   X_ch(i) += sum_q (C0_ch[q] + di C1_ch[q]) y_link[i + off + q].
// The filters are formed once per block from the terms' fractions, and a
// sample costs four multiply-adds per tap of its six links instead of the
// 32-weight construction per term.  Blocks outside these bounds (drift above
// 1e-4 samples, curvature of the delay above 1e-8 samples, a filter longer
// than kCombMax, a window too short) take the per-sample weights.
//
// Organisation: one CTA per group of G tiles (one FP64 set-up: the light-time
// polynomials at the group centre and the exact split of every term's delay
// there); the group is processed in sub-blocks of two tiles, each thread
// computing two samples 256 apart, so every coefficient read serves two
// samples.  The weights and their eps-derivatives come from warp-wide
// prefix and suffix products of dual numbers (d, d') = (eps + 15 - p, 1) over
// the 32 lanes: w_p = K_p prod_{m != p} d_m, w'_p its derivative.
#pragma once

#include "tdi_tile.cuh"

namespace lisa {


constexpr int kCombMax = 96;              // taps of one link's combined filter
constexpr int kSub = 2 * kTile;           // samples per sub-block
constexpr int kWinC = kSub + 256;         // staged link window per sub-block
constexpr unsigned kFull = 0xffffffffu;

struct CombSmem {
    double Tb[6][8];          // light-time polynomials around the group centre (FP64)
    int64_t J[48];            // group-centre split of each term's delay (term index ch * nterm + q)
    float f[48];
    Cubic dD[48];             // in-group variation of each term's delay (s)
    float Kc[32];             // Lagrange constants K_p
    int tw[6][8];             // per link: its terms
    int tsel[6][8];           // 0: the link's first channel, 1: its second
    float tsg[6][8];          // sign of the term
    int ntw[6];
    // per sub-block
    int64_t Jt[48];           // stencil centre of each term at the sub-block centre
    float ft[48], at[48];     // fraction there and its drift per sample
    int toff[6][8];
    int base0[6], L[6], wsh[6];   // wsh: link window shifted back by 0 or 1 so that base0 is even
    int64_t wlo;
    int wlen;
    float2 wt[48][32];
    float4 coef[6][kCombMax];
    alignas(8) float win[6][kWinC + 2];
    float inv_half, inv_dt, barg_c, barg_d;
};

__device__ __forceinline__ int comb_link_cha(int ls) { return ls < 2 ? 1 : 0; }

#ifndef LISA_COMB_CPASYNC
#define LISA_COMB_CPASYNC 1   // link windows filled by asynchronous 4-byte copies
#endif

// 4-byte asynchronous global -> shared copy; n (0 or 4) bytes are read and the
// rest of the word is zero-filled.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int n)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Per-sample weights (blocks outside the combined filters' bounds): the
// delays from the group-centre split and cubic, stencils from the window or
// from global memory.  Out of line.
static __device__ __noinline__ void comb_exact_sample(const TdiArgs& a, const CombSmem& s, int64_t ic, int64_t i,
                                               float (&acc)[3])
{
    const float* __restrict__ yg = (const float*)a.y;
    const int dm = (int)(i - ic);
    const float u = (float)dm * s.inv_half;
    acc[0] = acc[1] = acc[2] = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        for (int q = 0; q < a.nterm; ++q) {
            const int w = ch * a.nterm + q;
            const float v = s.f[w] - s.dD[w](u) * s.inv_dt;
            const float fv = floorf(v);
            const int64_t j = s.J[w] + dm + (int)fv;
            const float eps = v - fv;
            const TdiTerm& tm = c_terms[q];
            const int ls = c_cyc[ch][tm.link];
            const float val = interp_one<float>(s.win[ls], s.wlo - s.wsh[ls], s.wlen + s.wsh[ls],
                                                yg + (int64_t)ls * a.ny, a.ym.n_in, j, eps);
            acc[ch] += tm.sign > 0 ? val : -val;
        }
    }
}

// One group of nt tiles from tile t0 (group centre t0 kTile + G kTile / 2):
// the combined filters of each sub-block of two tiles, stored with the blend
// of the arguments.  Every thread must call it.
static __device__ void comb_group(const TdiArgs& a, int64_t t0, int nt, int G, CombSmem& s)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nw = 3 * a.nterm;
    const int64_t ic = t0 * kTile + (int64_t)G * kTile / 2;   // group centre
    const float* __restrict__ yg = (const float*)a.y;

    // (1) light-time polynomials at the group centre, constants
    {
        int64_t sg = ic / a.tab.S;
        if (sg >= a.tab.nseg) sg = a.tab.nseg - 1;
        if (sg < 0) sg = 0;
        const double half = 0.5 * a.tab.S;
        const double xc = ((double)(ic - sg * a.tab.S) - half) / half;
        if (t < 6) {
            double b[7];
            taylor_shift7(a.tab.coef + (sg * kNQ + kQT + t) * kNC, xc, b);
            for (int p = 0; p < 7; ++p) s.Tb[t][p] = b[p];
        }
        if (t >= 32 && t < 64) s.Kc[t - 32] = (float)lagrange32_k(t - 32);
        if (t == 64) {
            s.inv_half = (float)(2.0 / a.tab.S);
            s.inv_dt = (float)(1.0 / a.ym.dt_in);
            const double tc = a.t0_out + (double)ic * a.dt_out;
            s.barg_c = (float)(a.bl.enabled ? a.bl.eps * (tc - a.bl.t_hyb) / a.bl.sigma : 0.0);
            s.barg_d = (float)(a.bl.enabled ? a.bl.eps * a.dt_out / a.bl.sigma : 0.0);
        }
        if (t >= 96 && t < 102) {
            // the terms of link ls, which enters channels (cha, chb)
            const int ls = t - 96;
            int n = 0;
            for (int ch = 0; ch < 3; ++ch)
                for (int q = 0; q < a.nterm; ++q)
                    if (c_cyc[ch][c_terms[q].link] == ls && n < 8) {
                        s.tw[ls][n] = ch * a.nterm + q;
                        s.tsel[ls][n] = ch == comb_link_cha(ls) ? 0 : 1;
                        s.tsg[ls][n] = c_terms[q].sign > 0 ? 1.f : -1.f;
                        ++n;
                    }
            s.ntw[ls] = n;
        }
    }
    __syncthreads();
    // (2) each term's delay at the group centre, split exactly (FP64), and its
    // in-group variation as an FP32 cubic
    if (t < nw) {
        const int ch = t / a.nterm, q = t % a.nterm;
        const TdiTerm& tm = c_terms[q];
        double Dc = 0.0;
        double c1 = 0.0, c2 = 0.0, c3 = 0.0;
        for (int k = 0; k < tm.nd; ++k) {
            const int li = c_cyc[ch][tm.d[k]];
            Dc += s.Tb[li][0];
            c1 += s.Tb[li][1];
            c2 += s.Tb[li][2];
            c3 += s.Tb[li][3];
        }
        int64_t j;
        double eps;
        split_f64(a.ym, ic, Dc, j, eps);
        s.J[t] = j;
        s.f[t] = (float)eps;
        s.dD[t] = Cubic{(float)c1, (float)c2, (float)c3};
    }
    __syncthreads();

    const float ih = s.inv_half, idt = s.inv_dt;
    for (int sb = 0; sb < nt; sb += 2) {
        const int64_t i0 = (t0 + sb) * (int64_t)kTile;
        const int64_t ipc = i0 + kTile;            // sub-block centre
        const int dti = (int)(ipc - ic);
        // (3) each term at the sub-block centre: stencil centre, fraction,
        // drift per sample; bounds of the linearisation
        bool good = true;
        if (t < nw) {
            const Cubic cv = s.dD[t];
            const float uc = (float)dti * ih;
            const float v = s.f[t] - cv(uc) * idt;
            const float fv = floorf(v);
            s.Jt[t] = s.J[t] + dti + (int)fv;
            s.ft[t] = v - fv;
            const float d1 = fmaf(uc, fmaf(3.f * cv.c3, uc, 2.f * cv.c2), cv.c1);   // dD/du at uc
            const float aw = -d1 * ih * idt;
            const float bw = -fmaf(3.f * cv.c3, uc, cv.c2) * ih * ih * idt;
            const float cw = -cv.c3 * ih * ih * ih * idt;
            const float h = 0.5f * kSub;
            good = fabsf(aw) * h <= 1e-4f && fabsf(bw) * h * h + fabsf(cw) * h * h * h <= 1e-8f;
            s.at[t] = aw;
        }
        good = __syncthreads_and(good);
        // (4) window: every term's stencils for di in [-kTile, kTile)
        if (warp == 0) {
            int64_t lo = INT64_MAX, hi = INT64_MIN;
            for (int w = lane; w < nw; w += 32) {
                lo = min(lo, s.Jt[w]);
                hi = max(hi, s.Jt[w]);
            }
            for (int off = 16; off > 0; off >>= 1) {
                lo = min(lo, (int64_t)__shfl_xor_sync(kFull, (long long)lo, off));
                hi = max(hi, (int64_t)__shfl_xor_sync(kFull, (long long)hi, off));
            }
            if (lane == 0) {
                s.wlo = lo - kTile - 15 - 2;
                const int64_t len = (hi + kTile - 1 + 16 + 2) - s.wlo + 1;
                s.wlen = len <= kWinC ? (int)len : 0;
            }
        }
        __syncthreads();
        const int64_t wlo = s.wlo;
        const int wlen = s.wlen;
        // (5) link filters: offsets and lengths
        if (t < 6) {
            const int ls = t;
            int64_t jlo = INT64_MAX, jhi = INT64_MIN;
            for (int r = 0; r < s.ntw[ls]; ++r) {
                jlo = min(jlo, s.Jt[s.tw[ls][r]]);
                jhi = max(jhi, s.Jt[s.tw[ls][r]]);
            }
            for (int r = 0; r < s.ntw[ls]; ++r) s.toff[ls][r] = (int)(s.Jt[s.tw[ls][r]] - jlo);
            const int64_t L = ((jhi - jlo + 32) + 3) / 4 * 4;
            const int64_t b0 = jlo - 15 - wlo;
            // samples di in [-kTile, kTile) read [b0 + di, b0 + di + L)
            if (wlen == 0 || L > kCombMax || b0 - kTile < 0 || b0 + kTile - 1 + L > wlen) good = false;
            s.L[ls] = (int)(L < kCombMax ? L : kCombMax);
            // the link's window starts one sample earlier when b0 is odd, so
            // that a thread's tap pairs (two adjacent samples) are 8-byte aligned
            const int sh = (int)(b0 & 1);
            s.wsh[ls] = sh;
            s.base0[ls] = (int)b0 + sh;
        }
        good = __syncthreads_and(good);
        // link windows: y on [wlo - wsh, wlo - wsh + wlen + 2) (the last two
        // entries only feed the unused half of a thread's last tap pair)
        // (asynchronous copies complete before the barrier ahead of the filters,
        // overlapping the weights and coefficients below)
        for (int li = 0; li < 6; ++li) {
            const int64_t org = wlo - s.wsh[li];
            const float* __restrict__ yl = yg + (int64_t)li * a.ny;
            for (int o = t; o < wlen + 2; o += blockDim.x) {
                const int64_t idx = org + o;
                const bool in = idx >= 0 && idx < a.ym.n_in;
#if LISA_COMB_CPASYNC
                cp_async4(&s.win[li][o], in ? yl + idx : yl, in ? 4 : 0);
#else
                s.win[li][o] = in ? yl[idx] : 0.f;
#endif
            }
        }
        // (6) weights and eps-derivatives: one warp per term, lane p
        if (good) {
            for (int w = warp; w < nw; w += kTile / 32) {
                const float e = s.ft[w];
                float pv = e + (float)(15 - lane), pd = 1.f;      // inclusive prefix product (dual)
                float sv = pv, sd = 1.f;                            // inclusive suffix product
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float bv = __shfl_up_sync(kFull, pv, off), bd = __shfl_up_sync(kFull, pd, off);
                    const float cv = __shfl_down_sync(kFull, sv, off), cd = __shfl_down_sync(kFull, sd, off);
                    if (lane >= off) {
                        pd = fmaf(pd, bv, pv * bd);
                        pv *= bv;
                    }
                    if (lane + off < 32) {
                        sd = fmaf(sd, cv, sv * cd);
                        sv *= cv;
                    }
                }
                float Pv = __shfl_up_sync(kFull, pv, 1), Pd = __shfl_up_sync(kFull, pd, 1);
                float Sv = __shfl_down_sync(kFull, sv, 1), Sd = __shfl_down_sync(kFull, sd, 1);
                if (lane == 0) { Pv = 1.f; Pd = 0.f; }
                if (lane == 31) { Sv = 1.f; Sd = 0.f; }
                const float K = s.Kc[lane];
                s.wt[w][lane] = make_float2(K * (Pv * Sv), K * fmaf(Pd, Sv, Pv * Sd));
            }
        }
        __syncthreads();
        // (7) combined coefficients
        if (good) {
            for (int k = t; k < 6 * kCombMax; k += blockDim.x) {
                const int ls = k / kCombMax, q = k % kCombMax;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < s.L[ls]) {
                    for (int r = 0; r < s.ntw[ls]; ++r) {
                        const int p = q - s.toff[ls][r];
                        if (p < 0 || p >= 32) continue;
                        const int w = s.tw[ls][r];
                        const float2 wv = s.wt[w][p];
                        const float c0 = s.tsg[ls][r] * wv.x, c1 = s.tsg[ls][r] * s.at[w] * wv.y;
                        if (s.tsel[ls][r] == 0) {
                            v.x += c0;
                            v.y += c1;
                        } else {
                            v.z += c0;
                            v.w += c1;
                        }
                    }
                }
                s.coef[ls][q] = v;
            }
        }
#if LISA_COMB_CPASYNC
        cp_async_wait_all();
#endif
        __syncthreads();
        // (8) samples i0 + 2t and i0 + 2t + 1 (block offsets di = 2t - kTile and
        // one more): the second sample's stencil is the first's shifted by one,
        // so the window is read as aligned pairs, each feeding both samples
        float X0[3], X1[3];
        if (good) {
            float a0[3] = {0.f, 0.f, 0.f}, a1[3] = {0.f, 0.f, 0.f};
            const float d0 = (float)(2 * t - kTile), d1 = d0 + 1.f;
#pragma unroll 1
            for (int ls = 0; ls < 6; ++ls) {
                const float2* __restrict__ yp =
                    reinterpret_cast<const float2*>(s.win[ls] + s.base0[ls] + (2 * t - kTile));
                const float4* __restrict__ cf = s.coef[ls];
                const int L = s.L[ls];
                float pa0 = 0.f, pa1 = 0.f, pb0 = 0.f, pb1 = 0.f;   // sample 0: channel a value/drift, b
                float qa0 = 0.f, qa1 = 0.f, qb0 = 0.f, qb1 = 0.f;   // sample 1
                float2 P = yp[0];
                for (int q = 0; q < L; q += 4) {
#pragma unroll
                    for (int k = 0; k < 4; k += 2) {
                        const float2 Pn = yp[(q + k) / 2 + 1];
                        const float4 c0 = cf[q + k], c1 = cf[q + k + 1];
                        // tap q + k: sample 0 reads P.x, sample 1 P.y
                        pa0 = fmaf(c0.x, P.x, pa0);
                        pa1 = fmaf(c0.y, P.x, pa1);
                        pb0 = fmaf(c0.z, P.x, pb0);
                        pb1 = fmaf(c0.w, P.x, pb1);
                        qa0 = fmaf(c0.x, P.y, qa0);
                        qa1 = fmaf(c0.y, P.y, qa1);
                        qb0 = fmaf(c0.z, P.y, qb0);
                        qb1 = fmaf(c0.w, P.y, qb1);
                        // tap q + k + 1: sample 0 reads P.y, sample 1 Pn.x
                        pa0 = fmaf(c1.x, P.y, pa0);
                        pa1 = fmaf(c1.y, P.y, pa1);
                        pb0 = fmaf(c1.z, P.y, pb0);
                        pb1 = fmaf(c1.w, P.y, pb1);
                        qa0 = fmaf(c1.x, Pn.x, qa0);
                        qa1 = fmaf(c1.y, Pn.x, qa1);
                        qb0 = fmaf(c1.z, Pn.x, qb0);
                        qb1 = fmaf(c1.w, Pn.x, qb1);
                        P = Pn;
                    }
                }
                const float va0 = fmaf(d0, pa1, pa0), vb0 = fmaf(d0, pb1, pb0);
                const float va1 = fmaf(d1, qa1, qa0), vb1 = fmaf(d1, qb1, qb0);
                // link ls enters channels (1, 2) for ls < 2, (0, 2) for ls < 4, else (0, 1)
                a0[0] += ls < 2 ? 0.f : va0;
                a0[1] += ls < 2 ? va0 : (ls < 4 ? 0.f : vb0);
                a0[2] += ls < 4 ? vb0 : 0.f;
                a1[0] += ls < 2 ? 0.f : va1;
                a1[1] += ls < 2 ? va1 : (ls < 4 ? 0.f : vb1);
                a1[2] += ls < 4 ? vb1 : 0.f;
            }
            for (int c = 0; c < 3; ++c) {
                X0[c] = a0[c];
                X1[c] = a1[c];
            }
        }
        // a sub-block of one tile (the group's last) has samples on t < kTile / 2 only
        if (sb + 1 < nt || 2 * t < kTile) {
            for (int r = 0; r < 2; ++r) {
                const int64_t i = i0 + 2 * t + r;
                if (i < a.i_begin || i >= a.i_end) continue;
                float X[3];
                if (good) {
                    for (int c = 0; c < 3; ++c) X[c] = r ? X1[c] : X0[c];
                } else {
                    comb_exact_sample(a, s, ic, i, X);
                }
                store_channels_f32(X[0], X[1], X[2], a.channels, a.bl, s.barg_c, s.barg_d, (int)(i - ic), i,
                                   (float*)a.xyz, a.nout);
            }
        }
        __syncthreads();   // the sub-block's shared data are reused by the next one
    }
}

}  // namespace lisa
