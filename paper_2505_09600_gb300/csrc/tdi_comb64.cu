// Michelson TDI 1.5 / 2.0 (Sec. II B, Eqs. X1.5, X2.0), FP64, frozen delays,
// link and output series on one sample grid: per-link combined filters.
//
// Each TDI term delays one link series by a sum of light times taken at the
// output time (the frozen form).  Over a sub-block of SB <= 512 consecutive
// output samples centred at ipc, the retarded position of term w at block
// offset di is
//   x_w(di) = J_w + di + f_w + delta_w(di),
//   delta_w(di) = a_w di + b_w di^2 + c_w di^3   (samples; the light times'
// Taylor series at ipc, the u^4 term below 1e-16 s),
// with (J_w, f_w) the exact FP64 split at ipc.  The light times change at
// |dL/dt|/c ~ 2e-8 (1 % arm flexing over a year), so |a_w di| stays below
// ~5e-5 and the term's 32 Lagrange weights are, to third order in delta,
//   w_p(f + delta) = T0_p + T1_p delta + T2_p delta^2 + T3_p delta^3,
// T_k the Taylor coefficients of w_p at f (sum_p |T1| < 3.7, |T2| < 4.3,
// |T3| < 3.8 over eps in [-0.05, 1.05]).  Collected by powers of di:
//   di^0: T0,  di^1: a T1,  di^2: b T1 + a^2 T2,  di^3: c T1 + 2ab T2 + a^3 T3.
// All terms that delay the same link add up to one filter of (spread of
// their delays + 32) taps with four coefficients per tap for each of the two
// channels the link enters (X: links 2..5, Y: 0, 1, 4, 5, Z: 0..3):
//   X_ch(i) += sum_q (C0[q] + di C1[q] + di^2 C2[q] + di^3 C3[q]) y[i + off + q].
// C0 and C1 and their tap sums are FP64.  The di^2 and di^3 parts are at most
// ~3e-8 of the link values (|b di^2| < 4e-9, |a di| < 5e-5), so they are
// formed and summed in FP32 (error below 1e-14 of the link values) from an
// FP32 copy of the window: a sample costs four FP64 multiply-adds per tap of
// its six links (GB300's FP64 pipe runs at 1/64 of the FP32 rate) instead of
// the 32-weight FP64 construction per term.  The dropped fourth-order terms
// are below 2e-14 of the link values under the bounds checked per sub-block
// (|a| h <= 1e-4, |b| h^2 <= 2e-8, |c| h^3 <= 1e-11, h = SB/2); a sub-block
// outside them, or whose filters or window do not fit, takes the per-sample
// FP64 path (the exact delay of every term and its own 32 weights).
//
// Organisation: one CTA per sub-block.  Warps 0..5 form the coefficients of
// one link each: per term, T0 and T1 by warp-wide prefix and suffix products
// of dual numbers (d, d') = (eps + 15 - p, 1) in FP64, T2 and T3 by the
// lane's own running product in FP32.  Thread t then takes the adjacent
// samples 2t and 2t + 1 of the block (one aligned pair load feeds both) for a
// slice of every link's taps; short ranges use small sub-blocks whose taps are
// split over 512 / SB slices, the slices' channel values summed in shared
// memory.
#include <cstdlib>

#include "tdi_tile.cuh"

namespace lisa {

constexpr int kC64Taps = 96;                   // taps of one link's combined filter
constexpr int kC64Sub = 512;                   // largest sub-block
constexpr int kC64Win = kC64Sub + kC64Taps + 8;   // staged link window (even)
constexpr unsigned kC64Full = 0xffffffffu;

struct C64Coef {
    double c0a, c1a, c0b, c1b;   // FP64 value and di coefficients, channel a then b
    float c2a, c3a, c2b, c3b;    // FP32 di^2 and di^3 coefficients
};

struct Comb64Smem {
    double Tb[6][8];             // light time of each link around ipc, polynomial in u = di / half (s)
    double Kd[32];               // Lagrange constants K_p
    int64_t J[48];               // split of each term's delay at ipc
    double f[48];
    double ca[48], cb[48], cc[48];   // delta(di) = ca di + cb di^2 + cc di^3
    int tw[6][8];                // per link: its terms
    int tsel[6][8];              // 0: the link's first channel, 1: its second
    float tsg[6][8];             // sign of the term
    int ntw[6];
    int toff[6][8];
    int base0[6], L[6], wsh[6];  // wsh: link window shifted back by 0 or 1 so that base0 is even
    int64_t wlo;
    int wlen;
    alignas(16) C64Coef coef[6][kC64Taps];
    alignas(16) double win[6][kC64Win + 2];
    alignas(16) float winf[6][kC64Win + 2];
    double red[3][kC64Sub];      // channel values of the tap slices (slices > 1)
};

__device__ __forceinline__ int c64_link_cha(int ls) { return ls < 2 ? 1 : 0; }

// 8-byte asynchronous global -> shared copy; n (0 or 8) bytes are read and
// the rest zero-filled.
__device__ __forceinline__ void cp_async8(double* dst, const double* src, int n)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all64() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// X, Y, Z at sample i = ipc + di from the exact FP64 delay of every term (the
// light-time polynomials around ipc, full degree) and its own 32 weights;
// stencils from the window when it holds them, else from global memory.
static __device__ __noinline__ void c64_exact_sample(const TdiArgs& a, const Comb64Smem& s, int64_t i, int di,
                                                     double half, double (&acc)[3])
{
    const double* __restrict__ yg = (const double*)a.y;
    const double u = (double)di / half;
    double T[6];
    for (int li = 0; li < 6; ++li) T[li] = horner_d<7>(s.Tb[li], u);
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        for (int q = 0; q < a.nterm; ++q) {
            const TdiTerm& tm = c_terms[q];
            double D = 0.0;
            for (int k = 0; k < tm.nd; ++k) D += T[c_cyc[ch][tm.d[k]]];
            int64_t j;
            double eps;
            split_f64(a.ym, i, D, j, eps);
            const int ls = c_cyc[ch][tm.link];
            const double v = interp_one<double>(s.win[ls], s.wlo - s.wsh[ls], s.wlen + s.wsh[ls],
                                                yg + (int64_t)ls * a.ny, a.ym.n_in, j, eps);
            acc[ch] += tm.sign > 0 ? v : -v;
        }
    }
}

// T0 and T1 of link ls's term r (lane p): the leave-one-out product of the
// duals (eps + 15 - m, 1) by warp-wide prefix and suffix products.
__device__ __forceinline__ void c64_weights_f64(double e, int lane, double K, double& T0, double& T1)
{
    double pv = e + (double)(15 - lane), pd = 1.0;   // inclusive prefix product (dual)
    double sv = pv, sd = 1.0;                          // inclusive suffix product
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double bv = __shfl_up_sync(kC64Full, pv, off), bd = __shfl_up_sync(kC64Full, pd, off);
        const double cv = __shfl_down_sync(kC64Full, sv, off), cd = __shfl_down_sync(kC64Full, sd, off);
        if (lane >= off) {
            pd = fma(pd, bv, pv * bd);
            pv *= bv;
        }
        if (lane + off < 32) {
            sd = fma(sd, cv, sv * cd);
            sv *= cv;
        }
    }
    double Pv = __shfl_up_sync(kC64Full, pv, 1), Pd = __shfl_up_sync(kC64Full, pd, 1);
    double Sv = __shfl_down_sync(kC64Full, sv, 1), Sd = __shfl_down_sync(kC64Full, sd, 1);
    if (lane == 0) {
        Pv = 1.0;
        Pd = 0.0;
    }
    if (lane == 31) {
        Sv = 1.0;
        Sd = 0.0;
    }
    T0 = K * (Pv * Sv);
    T1 = K * fma(Pd, Sv, Pv * Sd);
}

// T2 and T3 (FP32): the lane's running product of the 31 factors
// (eps + 15 - m + delta), m != p, as a cubic in delta.
__device__ __forceinline__ void c64_weights_hi(float e, int lane, float K, float& T2, float& T3)
{
    float t0 = 1.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if (m == lane) continue;
        const float x = e + (float)(15 - m);
        t3 = fmaf(t3, x, t2);
        t2 = fmaf(t2, x, t1);
        t1 = fmaf(t1, x, t0);
        t0 *= x;
    }
    T2 = K * t2;
    T3 = K * t3;
}

__global__ void __launch_bounds__(256, 2) tdi_comb64_kernel(TdiArgs a, int SB, int force_exact)
{
    extern __shared__ __align__(16) unsigned char c64_raw[];
    Comb64Smem& s = *reinterpret_cast<Comb64Smem*>(c64_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nw = 3 * a.nterm;
    const int h = SB / 2;
    const int64_t sb0 = a.i_begin + (int64_t)blockIdx.x * SB;
    const int64_t ipc = sb0 + h;
    const double half = 0.5 * a.tab.S;
    const double* __restrict__ yg = (const double*)a.y;

    // (1) light-time polynomials around ipc, constants, the terms of each link
    {
        int64_t sg = ipc / a.tab.S;
        if (sg >= a.tab.nseg) sg = a.tab.nseg - 1;
        if (sg < 0) sg = 0;
        const double xc = ((double)(ipc - sg * a.tab.S) - half) / half;
        if (t < 6) {
            double b[7];
            taylor_shift7(a.tab.coef + (sg * kNQ + kQT + t) * kNC, xc, b);
            for (int p = 0; p < 7; ++p) s.Tb[t][p] = b[p];
            s.Tb[t][7] = 0.0;
        }
        if (t >= 32 && t < 64) s.Kd[t - 32] = lagrange32_k(t - 32);
        if (t >= 96 && t < 102) {
            // the terms of link ls, which enters channels (cha, chb)
            const int ls = t - 96;
            int n = 0;
            for (int ch = 0; ch < 3; ++ch)
                for (int q = 0; q < a.nterm; ++q)
                    if (c_cyc[ch][c_terms[q].link] == ls && n < 8) {
                        s.tw[ls][n] = ch * a.nterm + q;
                        s.tsel[ls][n] = ch == c64_link_cha(ls) ? 0 : 1;
                        s.tsg[ls][n] = c_terms[q].sign > 0 ? 1.f : -1.f;
                        ++n;
                    }
            s.ntw[ls] = n;
        }
    }
    __syncthreads();
    // (2) each term's delay at ipc, split exactly, and its Taylor coefficients
    // in di (the light times' polynomials are in u = di / half)
    bool good = true;
    if (t < nw) {
        const int ch = t / a.nterm, q = t % a.nterm;
        const TdiTerm& tm = c_terms[q];
        double D0 = 0.0, D1 = 0.0, D2 = 0.0, D3 = 0.0;
        for (int k = 0; k < tm.nd; ++k) {
            const int li = c_cyc[ch][tm.d[k]];
            D0 += s.Tb[li][0];
            D1 += s.Tb[li][1];
            D2 += s.Tb[li][2];
            D3 += s.Tb[li][3];
        }
        int64_t j;
        double eps;
        split_f64(a.ym, ipc, D0, j, eps);
        s.J[t] = j;
        s.f[t] = eps;
        const double r = 1.0 / half, idt = 1.0 / a.ym.dt_in;
        const double ca = -D1 * r * idt, cb = -D2 * r * r * idt, cc = -D3 * r * r * r * idt;
        s.ca[t] = ca;
        s.cb[t] = cb;
        s.cc[t] = cc;
        const double hh = (double)h;
        good = fabs(ca) * hh <= 1e-4 && fabs(cb) * hh * hh <= 2e-8 && fabs(cc) * hh * hh * hh <= 1e-11
               && !force_exact;
    }
    good = __syncthreads_and(good);
    // (3) window: every term's stencils for di in [-h, h)
    if (warp == 0) {
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int w = lane; w < nw; w += 32) {
            lo = min(lo, s.J[w]);
            hi = max(hi, s.J[w]);
        }
        for (int off = 16; off > 0; off >>= 1) {
            lo = min(lo, (int64_t)__shfl_xor_sync(kC64Full, (long long)lo, off));
            hi = max(hi, (int64_t)__shfl_xor_sync(kC64Full, (long long)hi, off));
        }
        if (lane == 0) {
            s.wlo = lo - h - 15 - 2;
            const int64_t len = (hi + h - 1 + 16 + 2) - s.wlo + 1;
            s.wlen = len <= kC64Win ? (int)len : 0;
        }
    }
    __syncthreads();
    const int64_t wlo = s.wlo;
    const int wlen = s.wlen;
    // (4) link filters: offsets and lengths
    if (t < 6) {
        const int ls = t;
        int64_t jlo = INT64_MAX, jhi = INT64_MIN;
        for (int r = 0; r < s.ntw[ls]; ++r) {
            jlo = min(jlo, s.J[s.tw[ls][r]]);
            jhi = max(jhi, s.J[s.tw[ls][r]]);
        }
        for (int r = 0; r < s.ntw[ls]; ++r) s.toff[ls][r] = (int)(s.J[s.tw[ls][r]] - jlo);
        const int64_t L = ((jhi - jlo + 32) + 3) / 4 * 4;
        const int64_t b0 = jlo - 15 - wlo;
        // samples di in [-h, h) read [b0 + di, b0 + di + L)
        if (wlen == 0 || L > kC64Taps || b0 - h < 0 || b0 + h - 1 + L > wlen) good = false;
        s.L[ls] = (int)(L < kC64Taps ? L : kC64Taps);
        // the link's window starts one sample earlier when b0 is odd, so that
        // a thread's tap pairs (two adjacent samples) are 16-byte aligned
        const int sh = (int)(b0 & 1);
        s.wsh[ls] = sh;
        s.base0[ls] = (int)b0 + sh;
    }
    good = __syncthreads_and(good);
    // link windows: y on [wlo - wsh, wlo - wsh + wlen + 2) (the last two
    // entries only feed the unused half of a thread's last tap pair), by
    // asynchronous copies that overlap the coefficients below
    for (int li = 0; li < 6; ++li) {
        const int64_t org = wlo - s.wsh[li];
        const double* __restrict__ yl = yg + (int64_t)li * a.ny;
        for (int o = t; o < wlen + 2; o += blockDim.x) {
            const int64_t idx = org + o;
            const bool in = idx >= 0 && idx < a.ym.n_in;
            cp_async8(&s.win[li][o], in ? yl + idx : yl, in ? 8 : 0);
        }
    }
    // (5) coefficients: warp ls forms link ls's filter, one term after the
    // other (the lanes of a term write distinct taps).  The di^2 and di^3
    // coefficients are scaled by h^2 and h^3 (exact: h is a power of two) and
    // applied to v = di / h, which keeps their FP32 products with strain-sized
    // link values far from the FP32 underflow.
    if (good && warp < 6) {
        const int ls = warp;
        for (int q = lane; q < kC64Taps; q += 32) s.coef[ls][q] = C64Coef{0.0, 0.0, 0.0, 0.0, 0.f, 0.f, 0.f, 0.f};
        __syncwarp();
        const double K = s.Kd[lane];
        const float hf = (float)h;
        for (int r = 0; r < s.ntw[ls]; ++r) {
            const int w = s.tw[ls][r];
            double T0, T1;
            c64_weights_f64(s.f[w], lane, K, T0, T1);
            float T2, T3;
            c64_weights_hi((float)s.f[w], lane, (float)K, T2, T3);
            const float A = (float)s.ca[w] * hf, B = (float)s.cb[w] * hf * hf, C = (float)s.cc[w] * hf * hf * hf;
            const float T1f = (float)T1;
            const float sgf = s.tsg[ls][r];
            const double sg = (double)sgf;
            const double d0 = sg * T0, d1 = (sg * s.ca[w]) * T1;
            const float f2 = sgf * fmaf(B, T1f, A * A * T2);
            const float f3 = sgf * fmaf(C, T1f, fmaf(2.f * A * B, T2, A * A * A * T3));
            C64Coef& c = s.coef[ls][s.toff[ls][r] + lane];
            if (s.tsel[ls][r] == 0) {
                c.c0a += d0;
                c.c1a += d1;
                c.c2a += f2;
                c.c3a += f3;
            } else {
                c.c0b += d0;
                c.c1b += d1;
                c.c2b += f2;
                c.c3b += f3;
            }
            __syncwarp();
        }
    }
    cp_async_wait_all64();
    __syncthreads();
    // the FP32 copy of the windows (the di^2, di^3 sums)
    for (int li = 0; li < 6; ++li)
        for (int o = t; o < wlen + 2; o += blockDim.x) s.winf[li][o] = (float)s.win[li][o];
    __syncthreads();

    // (6) taps: thread t takes samples k = 2 pair, 2 pair + 1 of the block
    // (di = k - h) for the taps of slice `slice` of every link
    const int np = h, nslice = 256 / np;
    const int pair = t % np, slice = t / np;
    const int di0 = 2 * pair - h;
    double X0[3] = {0.0, 0.0, 0.0}, X1[3] = {0.0, 0.0, 0.0};
    if (good) {
        const float v0 = (float)di0 / (float)h, v1 = (float)(di0 + 1) / (float)h;
#pragma unroll 1
        for (int ls = 0; ls < 6; ++ls) {
            const int L = s.L[ls];
            const int chunk = ((L + nslice - 1) / nslice + 1) & ~1;
            const int q0 = min(slice * chunk, L), q1 = min(q0 + chunk, L);
            const double2* __restrict__ yp = reinterpret_cast<const double2*>(s.win[ls] + s.base0[ls] + di0 + q0);
            const float2* __restrict__ yf = reinterpret_cast<const float2*>(s.winf[ls] + s.base0[ls] + di0 + q0);
            const C64Coef* __restrict__ cf = s.coef[ls] + q0;
            // sample 0: channel a value / di sums, channel b; sample 1 likewise
            double pa0 = 0.0, pa1 = 0.0, pb0 = 0.0, pb1 = 0.0, qa0 = 0.0, qa1 = 0.0, qb0 = 0.0, qb1 = 0.0;
            float pa2 = 0.f, pa3 = 0.f, pb2 = 0.f, pb3 = 0.f, qa2 = 0.f, qa3 = 0.f, qb2 = 0.f, qb3 = 0.f;
            if (q0 < q1) {
                double2 P = yp[0];
                float2 F = yf[0];
                for (int q = 0; q < q1 - q0; q += 2) {
                    const double2 Pn = yp[q / 2 + 1];
                    const float2 Fn = yf[q / 2 + 1];
                    const C64Coef c0 = cf[q], c1 = cf[q + 1];
                    // tap q: sample 0 reads P.x, sample 1 P.y
                    pa0 = fma(c0.c0a, P.x, pa0);
                    pa1 = fma(c0.c1a, P.x, pa1);
                    pb0 = fma(c0.c0b, P.x, pb0);
                    pb1 = fma(c0.c1b, P.x, pb1);
                    qa0 = fma(c0.c0a, P.y, qa0);
                    qa1 = fma(c0.c1a, P.y, qa1);
                    qb0 = fma(c0.c0b, P.y, qb0);
                    qb1 = fma(c0.c1b, P.y, qb1);
                    pa2 = fmaf(c0.c2a, F.x, pa2);
                    pa3 = fmaf(c0.c3a, F.x, pa3);
                    pb2 = fmaf(c0.c2b, F.x, pb2);
                    pb3 = fmaf(c0.c3b, F.x, pb3);
                    qa2 = fmaf(c0.c2a, F.y, qa2);
                    qa3 = fmaf(c0.c3a, F.y, qa3);
                    qb2 = fmaf(c0.c2b, F.y, qb2);
                    qb3 = fmaf(c0.c3b, F.y, qb3);
                    // tap q + 1: sample 0 reads P.y, sample 1 Pn.x
                    pa0 = fma(c1.c0a, P.y, pa0);
                    pa1 = fma(c1.c1a, P.y, pa1);
                    pb0 = fma(c1.c0b, P.y, pb0);
                    pb1 = fma(c1.c1b, P.y, pb1);
                    qa0 = fma(c1.c0a, Pn.x, qa0);
                    qa1 = fma(c1.c1a, Pn.x, qa1);
                    qb0 = fma(c1.c0b, Pn.x, qb0);
                    qb1 = fma(c1.c1b, Pn.x, qb1);
                    pa2 = fmaf(c1.c2a, F.y, pa2);
                    pa3 = fmaf(c1.c3a, F.y, pa3);
                    pb2 = fmaf(c1.c2b, F.y, pb2);
                    pb3 = fmaf(c1.c3b, F.y, pb3);
                    qa2 = fmaf(c1.c2a, Fn.x, qa2);
                    qa3 = fmaf(c1.c3a, Fn.x, qa3);
                    qb2 = fmaf(c1.c2b, Fn.x, qb2);
                    qb3 = fmaf(c1.c3b, Fn.x, qb3);
                    P = Pn;
                    F = Fn;
                }
            }
            const double d0 = (double)di0, d1 = d0 + 1.0;
            const double va0 = fma(d0, pa1, pa0) + (double)(v0 * v0 * fmaf(v0, pa3, pa2));
            const double vb0 = fma(d0, pb1, pb0) + (double)(v0 * v0 * fmaf(v0, pb3, pb2));
            const double va1 = fma(d1, qa1, qa0) + (double)(v1 * v1 * fmaf(v1, qa3, qa2));
            const double vb1 = fma(d1, qb1, qb0) + (double)(v1 * v1 * fmaf(v1, qb3, qb2));
            // link ls enters channels (1, 2) for ls < 2, (0, 2) for ls < 4, else (0, 1)
            X0[0] += ls < 2 ? 0.0 : va0;
            X0[1] += ls < 2 ? va0 : (ls < 4 ? 0.0 : vb0);
            X0[2] += ls < 4 ? vb0 : 0.0;
            X1[0] += ls < 2 ? 0.0 : va1;
            X1[1] += ls < 2 ? va1 : (ls < 4 ? 0.0 : vb1);
            X1[2] += ls < 4 ? vb1 : 0.0;
        }
        if (nslice > 1) {
            for (int c = 0; c < 3; ++c) {
                s.red[c][slice * SB + 2 * pair] = X0[c];
                s.red[c][slice * SB + 2 * pair + 1] = X1[c];
            }
        }
    }
    if (good && nslice > 1) {
        __syncthreads();
        if (t < SB) {
            double X[3];
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int sl = 0; sl < nslice; ++sl) v += s.red[c][sl * SB + t];
                X[c] = v;
            }
            const int64_t i = sb0 + t;
            if (i < a.i_end)
                store_channels<double>(X[0], X[1], X[2], a.channels, a.bl, a.t0_out, a.dt_out, i, (double*)a.xyz,
                                       a.nout);
        }
    } else if (good) {
        for (int r = 0; r < 2; ++r) {
            const int64_t i = sb0 + 2 * pair + r;
            if (i >= a.i_end) continue;
            const double* X = r ? X1 : X0;
            store_channels<double>(X[0], X[1], X[2], a.channels, a.bl, a.t0_out, a.dt_out, i, (double*)a.xyz,
                                   a.nout);
        }
    } else {
        for (int k = t; k < SB; k += blockDim.x) {
            const int64_t i = sb0 + k;
            if (i >= a.i_end) continue;
            double X[3];
            c64_exact_sample(a, s, i, k - h, half, X);
            store_channels<double>(X[0], X[1], X[2], a.channels, a.bl, a.t0_out, a.dt_out, i, (double*)a.xyz,
                                   a.nout);
        }
    }
}

// Launch over samples [a.i_begin, a.i_end) (host side): sub-blocks of 512
// samples, halved (down to 32, their taps split over more threads) while the
// range gives fewer than two CTAs per SM.  Coarse grids take shorter blocks:
// the delay's curvature term b h^2 grows as dt h^2 (about 4e-9 at dt = 5 s,
// h = 256), so h shrinks by 2 for every factor 4 in dt above 10 s.  The
// environment variable LISA_TDI64_EXACT=1 sends every sub-block through the
// per-sample path (tests).
int launch_tdi_comb64(const TdiArgs& a, cudaStream_t st)
{
    static int sms[64] = {0};
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    const int d = dev < 64 ? dev : 63;
    if (sms[d] == 0) {
        cudaDeviceGetAttribute(&sms[d], cudaDevAttrMultiProcessorCount, dev);
        if (sms[d] <= 0) sms[d] = 1;
    }
    if (!attr[d]) {
        const cudaError_t e = cudaFuncSetAttribute(tdi_comb64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(Comb64Smem));
        if (e != cudaSuccess) return cuda_status(e, "tdi_comb64_kernel shared memory");
        attr[d] = true;
    }
    const int64_t n = a.i_end - a.i_begin;
    int SB = kC64Sub;
    for (double dt = a.dt_out; dt > 10.0 && SB > 32; dt *= 0.25) SB >>= 1;
    while (SB > 32 && (n + SB - 1) / SB < 2 * (int64_t)sms[d]) SB >>= 1;
    const int64_t grid = (n + SB - 1) / SB;
    const char* ev = getenv("LISA_TDI64_EXACT");
    const int force_exact = (ev && ev[0] == '1') ? 1 : 0;
    tdi_comb64_kernel<<<(unsigned)grid, 256, sizeof(Comb64Smem), st>>>(a, SB, force_exact);
    return cuda_status(cudaGetLastError(), "tdi_comb64_kernel launch");
}

}  // namespace lisa
