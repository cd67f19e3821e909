// Likelihood tail of the response (Sec. IV, steps iv-v of the timing: the
// Fourier transform of A, E, T and the noise-weighted inner product,
// Eq. scalar_product), with the analytic A/E/T noise PSDs of Sec. II C
// (Eqs. SnAE, SnT, sgal).
//
//   lisa_psd_aet            S^{A,E}(f), S^T(f) on a frequency grid (FP64)
//   lisa_noise_weights_aet  w_k = 4 df / S(f_k) (FP64) on the rfft bins of a time
//                           grid inside [f_min, f_max], zero elsewhere (the
//                           rectangle rule of Eq. scalar_product; computed
//                           once per grid and reused by every inner product)
//   lisa_inner_aet          <x|y>, <x|x>, <y|y> per channel: the real FFTs of
//                           x and y (cuFFT, batched over the three rows), then
//                           one pass over the bins and a fixed-order
//                           reduction (deterministic)
// The continuous transform is dt times the discrete one, x~(f_k) =
// dt sum_n x_n exp(-2 pi i k n / N): the phase of the grid start cancels in
// x~^* y~, and the products carry dt^2.
#include <cufft.h>
#include <math.h>

#include <mutex>
#include <vector>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

namespace lisa {

namespace {

constexpr double kSacc = 2.4e-15 * 2.4e-15;    // m^2 s^-4 Hz^-1
constexpr double kSoms = 7.9e-12 * 7.9e-12;    // m^2 Hz^-1
constexpr double kGalA = 1.28265531e-44, kGalAlpha = 1.62966700, kGalF2 = 4.81078093e-4;
constexpr double kGalA1 = -0.223499956, kGalB1 = -2.70408439, kGalAk = -0.360976122, kGalBk = -2.37822436;

struct NoiseSpec {
    int gen, galaxy;
    double L, f1, fknee;
};

NoiseSpec make_spec(int tdi_gen, double L_m, double t_obs_years, int galaxy)
{
    const double lt = log10(t_obs_years);
    return NoiseSpec{tdi_gen, galaxy, L_m, pow(10.0, kGalA1 * lt + kGalB1), pow(10.0, kGalAk * lt + kGalBk)};
}

// S^{A,E} and S^T at frequency f (f > 0).
__device__ void psd_at(const NoiseSpec& ns, double f, double& sae, double& st)
{
    const double x = 2.0 * kPi * f * ns.L / kC;
    double sx, cx;
    sincos(x, &sx, &cx);
    const double w = 2.0 * kPi * f;
    const double r4 = 4e-4 / f, r8 = f / 8e-3, r2 = 2e-3 / f;
    const double pm = kSacc / (w * kC * w * kC) * (1.0 + r4 * r4) * (1.0 + r8 * r8 * r8 * r8);
    const double op = kSoms * (w / kC) * (w / kC) * (1.0 + r2 * r2 * r2 * r2);
    double gal = 0.0;
    if (ns.galaxy)
        gal = 2.0 * x * x * sx * sx * kGalA * pow(f, -7.0 / 3.0) * exp(-pow(f / ns.f1, kGalAlpha)) *
              (1.0 + tanh((ns.fknee - f) / kGalF2));
    const double s2x = 2.0 * sx * cx;                       // sin 2x
    const double lam = ns.gen == LISA_TDI20 ? 4.0 * s2x * s2x : 1.0;
    const double c2x = cx * cx - sx * sx;                   // cos 2x
    const double sh = sin(0.5 * x);
    sae = 8.0 * lam * sx * sx * (2.0 * (3.0 + 2.0 * cx + c2x) * pm + (2.0 + cx) * op) + 1.5 * lam * gal;
    st = 16.0 * lam * sx * sx * ((1.0 - cx) * op + 8.0 * sh * sh * sh * sh * pm) + lam * gal;
}

__global__ void psd_kernel(NoiseSpec ns, double f0, double df, int64_t nf, double* __restrict__ psd)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    double sae, st;
    psd_at(ns, f0 + (double)k * df, sae, st);
    psd[k] = sae;
    psd[nf + k] = st;
}

// Weights in FP64 for both forms: S_n is ~1e-44 (fractional frequency), so
// 4 df / S_n is far above the FP32 range.
// Bin frequency k / (M dt) by a division (the band test at f_min, f_max must
// not depend on how f_k was rounded: next to a PSD zero one bin's weight can
// dominate a product).
__global__ void weights_kernel(NoiseSpec ns, double span, int64_t nf, double f_min, double f_max, double* __restrict__ w)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const double f = (double)k / span;
    const double df = 1.0 / span;
    double wa = 0.0, wt = 0.0;
    if (k > 0 && f >= f_min && f <= f_max) {
        double sae, st;
        psd_at(ns, f, sae, st);
        wa = sae > 0.0 ? 4.0 * df / sae : 0.0;
        wt = st > 0.0 ? 4.0 * df / st : 0.0;
    }
    w[k] = wa;
    w[nf + k] = wt;
}

constexpr int kRedThreads = 256;
constexpr float kSc32 = 18446744073709551616.f;   // 2^64
constexpr float kLo32 = 2.0194839173657902e-28f;    // 2^-92

// The nine sums of one thread's grid-stride range of bins in FP64 (channel c:
// sum w Re(X* Y), sum w |X|^2, sum w |Y|^2).
template <typename Cplx>
__device__ __forceinline__ void inner_bins_f64(const Cplx* __restrict__ X, const Cplx* __restrict__ Y,
                                               const double* __restrict__ w, int64_t nf, double* acc)
{
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += (int64_t)gridDim.x * blockDim.x) {
        const double wa = w[k], wt = w[nf + k];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const Cplx a = X[(int64_t)c * nf + k], b = Y[(int64_t)c * nf + k];
            const double ww = c < 2 ? wa : wt;
            const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
            acc[3 * c + 0] = fma(ww, ax * bx + ay * by, acc[3 * c + 0]);
            acc[3 * c + 1] = fma(ww, ax * ax + ay * ay, acc[3 * c + 1]);
            acc[3 * c + 2] = fma(ww, bx * bx + by * by, acc[3 * c + 2]);
        }
    }
}

// FP32 spectra: on this part the FP64 pipe (which also converts between FP32 and
// FP64) runs far below the FP32 rate, so a bin's products, weighting and sums are
// formed in FP32 where the values allow, and the FP32 sums are added to FP64 ones
// every kFlush bins of a thread.
//  - Operands are scaled by 2^64: for max|component| in [2^-92, 2^-1) the scaled
//    squares and their sums are normal FP32 numbers. The weight carries the
//    scale 2^-128 and is used in FP32 when it is zero or in [2^-60, 2^61)
//    after scaling (converted with integer operations, off the FP64 pipe).
//  - A product with an operand or weight outside those ranges is formed in FP64.
//    Each square is decided by its own operand.
//  - A thread whose FP32 sums of squares of X (or of Y) reach 2^120 or overflow
//    recomputes those sums over its bins in FP64, and the cross sums with them
//    (the cross sums are bounded by the squares).  The sums of squares of the
//    other operand are kept, so <X|X> does not depend on Y.
constexpr int kFlush = 16;

// FP64 recomputation of a thread's bins for the sums selected: the squares of
// X (redo_x), of Y (redo_y) and the cross sums (either).
template <typename Cplx>
__device__ __noinline__ void inner_bins_redo_f64(const Cplx* __restrict__ X, const Cplx* __restrict__ Y,
                                                 const double* __restrict__ w, int64_t nf, bool redo_x, bool redo_y,
                                                 double* acc)
{
    double r[9];
    inner_bins_f64(X, Y, w, nf, r);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[3 * c + 0] = r[3 * c + 0];
        if (redo_x) acc[3 * c + 1] = r[3 * c + 1];
        if (redo_y) acc[3 * c + 2] = r[3 * c + 2];
    }
}

// w * 2^-128 as an FP32 number, formed from the bits of w with integer
// operations (round to nearest, ties away), for w == 0 or w * 2^-128 in
// [2^-60, 2^61); false for anything else (negative, NaN or out of range).
__device__ __forceinline__ bool weight_f32(double w, float& f)
{
    const long long bits = __double_as_longlong(w);
    const long long e = bits >> 52;                            // biased exponent (sign 0)
    const bool ok = bits == 0 || (e >= 1023 + 128 - 60 && e <= 1023 + 128 + 60);
    const long long r = ((bits + (1LL << 28)) >> 29) - (1024LL << 23);
    f = bits == 0 ? 0.f : __int_as_float((int)r);
    return ok;
}

__device__ __forceinline__ void inner_bins_f32(const float2* __restrict__ X, const float2* __restrict__ Y,
                                               const double* __restrict__ w, int64_t nf, double* acc)
{
    float s[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) { acc[q] = 0.0; s[q] = 0.f; }
    bool bad_x = false, bad_y = false;
    int cnt = 0;
    auto flush = [&]() {
        bool fine_x = true, fine_y = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fine_x = fine_x && s[3 * c + 1] < 1.329228e36f;
            fine_y = fine_y && s[3 * c + 2] < 1.329228e36f;
        }
        bad_x = bad_x || !fine_x;
        bad_y = bad_y || !fine_y;
#pragma unroll
        for (int q = 0; q < 9; ++q) { acc[q] += (double)s[q]; s[q] = 0.f; }
    };
    // the next bin's loads are issued before the current bin is formed (two bins in
    // flight per thread: the pass is bound by memory latency)
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float2 ca[3], cb[3];
    double wa = 0.0, wt = 0.0;
    if (k < nf) {
        wa = w[k];
        wt = w[nf + k];
#pragma unroll
        for (int c = 0; c < 3; ++c) { ca[c] = X[(int64_t)c * nf + k]; cb[c] = Y[(int64_t)c * nf + k]; }
    }
    for (; k < nf; k += step) {
        const int64_t kn = k + step;
        float2 na[3] = {}, nb[3] = {};
        double nwa = 0.0, nwt = 0.0;
        if (kn < nf) {
            nwa = w[kn];
            nwt = w[nf + kn];
#pragma unroll
            for (int c = 0; c < 3; ++c) { na[c] = X[(int64_t)c * nf + kn]; nb[c] = Y[(int64_t)c * nf + kn]; }
        }
        float fa, ft;
        const bool oka = weight_f32(wa, fa), okt = weight_f32(wt, ft);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 a = ca[c], b = cb[c];
            const bool okw = c < 2 ? oka : okt;
            const float wf = c < 2 ? fa : ft;
            const float mA = fmaxf(fabsf(a.x), fabsf(a.y)), mB = fmaxf(fabsf(b.x), fabsf(b.y));
            const bool okA = okw && mA >= kLo32 && mA < 0.5f, okB = okw && mB >= kLo32 && mB < 0.5f;
            const float ax = a.x * kSc32, ay = a.y * kSc32, bx = b.x * kSc32, by = b.y * kSc32;
            if (okA && okB) {
                s[3 * c + 0] = fmaf(wf, fmaf(ax, bx, ay * by), s[3 * c + 0]);
                s[3 * c + 1] = fmaf(wf, fmaf(ax, ax, ay * ay), s[3 * c + 1]);
                s[3 * c + 2] = fmaf(wf, fmaf(bx, bx, by * by), s[3 * c + 2]);
            } else {
                const double ww = c < 2 ? wa : wt;
                const double dax = a.x, day = a.y, dbx = b.x, dby = b.y;
                acc[3 * c + 0] = fma(ww, dax * dbx + day * dby, acc[3 * c + 0]);
                if (okA) s[3 * c + 1] = fmaf(wf, fmaf(ax, ax, ay * ay), s[3 * c + 1]);
                else acc[3 * c + 1] = fma(ww, dax * dax + day * day, acc[3 * c + 1]);
                if (okB) s[3 * c + 2] = fmaf(wf, fmaf(bx, bx, by * by), s[3 * c + 2]);
                else acc[3 * c + 2] = fma(ww, dbx * dbx + dby * dby, acc[3 * c + 2]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) { ca[c] = na[c]; cb[c] = nb[c]; }
        wa = nwa;
        wt = nwt;
        if (++cnt == kFlush) { flush(); cnt = 0; }
    }
    flush();
    if (bad_x || bad_y) inner_bins_redo_f64(X, Y, w, nf, bad_x, bad_y, acc);
}

// Per block: the nine sums over the block's threads, FP64 in a fixed-order tree.
template <typename Cplx>
__global__ void __launch_bounds__(kRedThreads, 3) inner_kernel(const Cplx* __restrict__ X, const Cplx* __restrict__ Y,
                                                            const double* __restrict__ w, int64_t nf,
                                                            double* __restrict__ partial)
{
    double acc[9];
    if constexpr (sizeof(X->x) == 4) inner_bins_f32(X, Y, w, nf, acc);
    else inner_bins_f64(X, Y, w, nf, acc);
    __shared__ double red[9][kRedThreads];
#pragma unroll
    for (int q = 0; q < 9; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 9; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 9) partial[(int64_t)blockIdx.x * 9 + threadIdx.x] = red[threadIdx.x][0];
}

// Sum of the block partials, times dt^2: warp q sums value q, lane l the blocks
// l, l + 32, ... in order, then a fixed butterfly (run-to-run identical).
__global__ void inner_finish_kernel(const double* __restrict__ partial, int nblocks, double dt2, double* __restrict__ out)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= 9) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(int64_t)b * 9 + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[q] = s * dt2;
}

// cuFFT plans (three real rows of n samples, batched), one per (device, n,
// precision), created on first use and kept for the process.
struct PlanEntry {
    int device;
    int64_t n;
    int precision;
    cufftHandle plan;
};
std::mutex g_plan_mutex;
std::vector<PlanEntry> g_plans;

int get_plan(int64_t n, int precision, cufftHandle& out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    for (const PlanEntry& e : g_plans)
        if (e.device == dev && e.n == n && e.precision == precision) {
            out = e.plan;
            return LISA_OK;
        }
    cufftHandle p;
    long long nn[1] = {(long long)n};
    size_t ws = 0;
    if (cufftCreate(&p) != CUFFT_SUCCESS) {
        set_error("cufftCreate failed");
        return LISA_ECUDA;
    }
    const cufftType type = precision == LISA_MIXED ? CUFFT_R2C : CUFFT_D2Z;
    const long long nf = n / 2 + 1;
    if (cufftMakePlanMany64(p, 1, nn, nullptr, 1, n, nullptr, 1, nf, type, 3, &ws) != CUFFT_SUCCESS) {
        cufftDestroy(p);
        set_error("cufftMakePlanMany64 failed for n = %lld", (long long)n);
        return LISA_ECUDA;
    }
    g_plans.push_back(PlanEntry{dev, n, precision, p});
    out = p;
    return LISA_OK;
}

int rfft3(cufftHandle plan, int precision, const void* in, void* out, cudaStream_t st)
{
    if (cufftSetStream(plan, st) != CUFFT_SUCCESS) { set_error("cufftSetStream failed"); return LISA_ECUDA; }
    cufftResult r;
    if (precision == LISA_MIXED) r = cufftExecR2C(plan, (cufftReal*)in, (cufftComplex*)out);
    else r = cufftExecD2Z(plan, (cufftDoubleReal*)in, (cufftDoubleComplex*)out);
    if (r != CUFFT_SUCCESS) { set_error("cuFFT execution failed (%d)", (int)r); return LISA_ECUDA; }
    return LISA_OK;
}

}  // namespace

}  // namespace lisa

using namespace lisa;

extern "C" {

int lisa_psd_aet(double f0, double df, int64_t nf, int tdi_gen, double L_m, double t_obs_years, int galaxy, double* psd,
                 void* stream)
{
    if (tdi_gen != LISA_TDI15 && tdi_gen != LISA_TDI20) { set_error("tdi_gen must be 15 or 20"); return LISA_EINVAL; }
    if (nf < 0 || !(f0 > 0.0) || !(df >= 0.0) || !(L_m > 0.0) || !(t_obs_years > 0.0)) {
        set_error("need f0 > 0, df >= 0, nf >= 0, L_m > 0, t_obs_years > 0");
        return LISA_EINVAL;
    }
    if (nf == 0) return LISA_OK;
    if (!psd) { set_error("psd is NULL"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    prof_before("psd_aet", st);
    psd_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(make_spec(tdi_gen, L_m, t_obs_years, galaxy), f0, df, nf,
                                                             psd);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "psd_kernel launch");
}

int64_t lisa_fft_length(int64_t n)
{
    if (n <= 1) return n < 1 ? 0 : 1;
    int64_t best = -1;
    for (int64_t p2 = 1; p2 < 2 * n; p2 *= 2)
        for (int64_t p3 = p2; p3 < 2 * n; p3 *= 3)
            for (int64_t p5 = p3; p5 < 2 * n; p5 *= 5)
                for (int64_t p7 = p5; p7 < 2 * n; p7 *= 7)
                    if (p7 >= n && (best < 0 || p7 < best)) best = p7;
    return best;
}

int lisa_noise_weights_aet(lisa_grid grid, int64_t nfft, int tdi_gen, double L_m, double t_obs_years, int galaxy,
                           double f_min, double f_max, double* w, void* stream)
{
    LISA_TRY(check_grid(grid, "grid"));
    if (nfft == 0) nfft = grid.n;
    if (nfft < grid.n) { set_error("nfft = %lld is below the grid's %lld samples", (long long)nfft, (long long)grid.n); return LISA_EINVAL; }
    if (tdi_gen != LISA_TDI15 && tdi_gen != LISA_TDI20) { set_error("tdi_gen must be 15 or 20"); return LISA_EINVAL; }
    if (!(L_m > 0.0) || !(t_obs_years > 0.0) || !(f_max >= f_min)) {
        set_error("need L_m > 0, t_obs_years > 0, f_max >= f_min");
        return LISA_EINVAL;
    }
    if (grid.n == 0) return LISA_OK;
    if (!w) { set_error("w is NULL"); return LISA_EINVAL; }
    const int64_t nf = nfft / 2 + 1;
    const double span = (double)nfft * grid.dt;   // M dt: f_k = k / span, df = 1 / span
    cudaStream_t st = (cudaStream_t)stream;
    const NoiseSpec ns = make_spec(tdi_gen, L_m, t_obs_years, galaxy);
    const unsigned blocks = (unsigned)((nf + 255) / 256);
    prof_before("noise_weights", st);
    weights_kernel<<<blocks, 256, 0, st>>>(ns, span, nf, f_min, f_max, w);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "weights_kernel launch");
}

int lisa_inner_aet(lisa_grid grid, int64_t nfft, const void* x, const void* y, int precision, const double* w,
                   double* out, void* stream)
{
    LISA_TRY(check_grid(grid, "grid"));
    if (precision != LISA_F64 && precision != LISA_MIXED) { set_error("precision unknown"); return LISA_EINVAL; }
    if (grid.n < 2) { set_error("need at least 2 samples"); return LISA_EINVAL; }
    if (!x || !y || !w || !out) { set_error("NULL pointer"); return LISA_EINVAL; }
    if (nfft == 0) nfft = grid.n;
    if (nfft < grid.n) { set_error("nfft = %lld is below the grid's %lld samples", (long long)nfft, (long long)grid.n); return LISA_EINVAL; }
    const int64_t n = grid.n, nf = nfft / 2 + 1;
    cudaStream_t st = (cudaStream_t)stream;
    cufftHandle plan;
    std::lock_guard<std::mutex> lock(g_plan_mutex);   // one plan object is bound to one stream at a time
    LISA_TRY(get_plan(nfft, precision, plan));
    const size_t cs = precision == LISA_MIXED ? sizeof(cufftComplex) : sizeof(cufftDoubleComplex);
    const size_t rs = real_size(precision);
    Scratch sc(st);
    // rows zero-padded to nfft samples (a 7-smooth length keeps the transform fast)
    auto padded = [&](const void* src) -> const void* {
        if (nfft == n) return src;
        char* p = (char*)sc.alloc(3 * (size_t)nfft * rs);
        if (!p) return nullptr;
        if (cudaMemcpy2DAsync(p, (size_t)nfft * rs, src, (size_t)n * rs, (size_t)n * rs, 3, cudaMemcpyDeviceToDevice,
                              st) != cudaSuccess ||
            cudaMemset2DAsync(p + (size_t)n * rs, (size_t)nfft * rs, 0, (size_t)(nfft - n) * rs, 3, st) != cudaSuccess)
            return nullptr;
        return p;
    };
    const void* xp = padded(x);
    const void* yp = (y == x) ? xp : padded(y);
    if (!xp || !yp) {
        if (sc.status()) return sc.status();
        return cuda_status(cudaGetLastError(), "zero padding");
    }
    void* X = sc.alloc(3 * (size_t)nf * cs);
    void* Y = (x == y) ? X : sc.alloc(3 * (size_t)nf * cs);
    int nblocks = 0;
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // one wave of resident blocks (a second, partial wave would idle most SMs)
        int per_sm = 0;
        if (precision == LISA_MIXED)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inner_kernel<float2>, kRedThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inner_kernel<double2>, kRedThreads, 0);
        nblocks = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        const int64_t need = (nf + kRedThreads - 1) / kRedThreads;
        if (need < nblocks) nblocks = (int)(need > 0 ? need : 1);
    }
    double* partial = (double*)sc.alloc((size_t)nblocks * 9 * sizeof(double));
    if (!X || !Y || !partial) return sc.status();
    prof_before("inner_aet", st);
    LISA_TRY(rfft3(plan, precision, xp, X, st));
    if (y != x) LISA_TRY(rfft3(plan, precision, yp, Y, st));
    if (precision == LISA_MIXED)
        inner_kernel<float2><<<nblocks, kRedThreads, 0, st>>>((const float2*)X, (const float2*)Y, w, nf, partial);
    else
        inner_kernel<double2><<<nblocks, kRedThreads, 0, st>>>((const double2*)X, (const double2*)Y, w, nf, partial);
    inner_finish_kernel<<<1, 9 * 32, 0, st>>>(partial, nblocks, grid.dt * grid.dt, out);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "inner_kernel launch");
}

}  // extern "C"
