// sh_inverse_static: spectral -> grid synthesis that allocates nothing.
//
// Same result as sh_inverse, but with no plan: the Gaussian latitudes, the
// associated Legendre functions and the FFT twiddles are computed on the
// device inside the call, and the only intermediate storage (the latitudes
// and the Fourier coefficients between the Legendre sums and the longitude
// FFTs) lives in the file-scope device array g_static_scratch below.  That
// array is part of the loaded module: every GPU that loads this library holds
// its kStaticScratchBytes until the process exits.
#include <cfloat>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace mlsdc {
namespace {

constexpr size_t kStaticScratchBytes = 4u << 20;  // 4 MiB
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticMaxHalfLat = 1024;
// layout: [mu, w for the northern latitudes: 2 * kStaticMaxHalfLat doubles]
//         [Fourier coefficients: nf * J * (R+1) complex]
constexpr size_t kStaticLatDoubles = 2 * kStaticMaxHalfLat;
constexpr size_t kStaticFourierMax = (kStaticScratchBytes - kStaticLatDoubles * sizeof(double)) / sizeof(double2);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Host-side device addresses of g_static_scratch, one per device.  Outside
// stream capture every call looks the address up again (a cudaDeviceReset
// reloads the module, and the array may then sit elsewhere); under capture
// the address recorded by the last uncaptured call on that device is used.
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {nullptr};

__device__ __forceinline__ double2 s_cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Gaussian latitudes (Newton on P_J) and weights of the northern half.
__global__ void k_static_latitudes(double* lat, int J) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J / 2) return;
    const double pi = 3.14159265358979323846;
    double x = cos(pi * (j + 0.75) / (J + 0.5));
    double p0 = 1.0, p1 = x, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        p0 = 1.0;
        p1 = x;
        for (int k = 2; k <= J; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = J * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        // relative stop: near the poles one ulp of x is ~1.1e-16, so an
        // absolute 1e-16 test could run every iteration of the O(J) loop
        if (fabs(dx) <= 4.0 * DBL_EPSILON * fabs(x)) break;
    }
    p0 = 1.0;
    p1 = x;
    for (int k = 2; k <= J; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    dp = J * (x * p1 - p0) / (x * x - 1.0);
    lat[j] = x;
    lat[kStaticMaxHalfLat + j] = 2.0 / ((1.0 - x * x) * dp * dp);
}

__device__ __forceinline__ double s_eps(int m, int n) {
    return n <= m ? 0.0 : sqrt((double(n) * n - double(m) * m) / (4.0 * double(n) * n - 1.0));
}

// One thread per (northern latitude, m, field): the Legendre sums with
// P^m_n evaluated by recurrence, split in even/odd n - m for the mirror
// latitude.  Writes every Fourier coefficient m <= R of both rows.
__global__ void k_static_synth(const double2* __restrict__ spec, const double* __restrict__ lat, double2* four,
                               int R, int J, int nc) {
    const int J2 = J / 2;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    const int fld = blockIdx.z;
    if (j >= J2) return;
    const double x = lat[j];
    const double s = sqrt(1.0 - x * x);
    double pmm = sqrt(0.5);
    for (int k = 1; k <= m; ++k) {
        pmm *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
        if (fabs(pmm) < 1e-300) pmm = 0.0;
    }
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const double2* c = spec + (size_t)fld * nc + off;
    double2 e = make_double2(0.0, 0.0), o = make_double2(0.0, 0.0);
    double pm1 = 0.0, pn = pmm;
    for (int n = m; n <= R; ++n) {
        const double2 cn = c[n - m];
        if (((n - m) & 1) == 0) {
            e.x = fma(pn, cn.x, e.x);
            e.y = fma(pn, cn.y, e.y);
        } else {
            o.x = fma(pn, cn.x, o.x);
            o.y = fma(pn, cn.y, o.y);
        }
        double pn1 = (x * pn - s_eps(m, n) * pm1) / s_eps(m, n + 1);
        if (fabs(pn1) < 1e-300) pn1 = 0.0;
        pm1 = pn;
        pn = pn1;
    }
    double2* F = four + (size_t)fld * J * (R + 1);
    F[(size_t)j * (R + 1) + m] = make_double2(e.x + o.x, e.y + o.y);
    F[(size_t)(J - 1 - j) * (R + 1) + m] = make_double2(e.x - o.x, e.y - o.y);
}

// One block per grid row: real inverse DFT of length I through a complex
// DFT of length I/2 over z_k = x_{2k} + i x_{2k+1} (radix-2, twiddles from sincospi).
__global__ void k_static_irfft(const double2* __restrict__ four, double* __restrict__ grid, int R, int I) {
    extern __shared__ double2 sz[];
    const int row = blockIdx.x;
    const int Hn = I / 2;
    int logH = 0;
    while ((1 << logH) < Hn) ++logH;
    const double2* F = four + (size_t)row * (R + 1);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) {
        double2 a = k == 0 ? make_double2(F[0].x, 0.0) : (k <= R ? F[k] : make_double2(0.0, 0.0));
        const int kc = Hn - k;
        double2 c = kc <= R ? F[kc] : make_double2(0.0, 0.0);  // kc >= 1
        c.y = -c.y;
        double sn, cs;
        sincospi(2.0 * k / I, &sn, &cs);
        const double2 d = s_cmul(make_double2(a.x - c.x, a.y - c.y), make_double2(cs, sn));
        const double2 sum = make_double2(a.x + c.x, a.y + c.y);
        const int r = (int)(__brev((unsigned)k) >> (32 - logH));
        sz[r] = make_double2(sum.x - d.y, sum.y + d.x);
    }
    __syncthreads();
    for (int st = 0; st < logH; ++st) {
        const int h = 1 << st;
        for (int b = threadIdx.x; b < Hn / 2; b += blockDim.x) {
            const int pos = b & (h - 1);
            const int i0 = ((b >> st) << (st + 1)) + pos;
            double sn, cs;
            sincospi((double)pos / h, &sn, &cs);  // exp(+i pi pos / h)
            const double2 u = sz[i0];
            const double2 v = s_cmul(sz[i0 + h], make_double2(cs, sn));
            sz[i0] = make_double2(u.x + v.x, u.y + v.y);
            sz[i0 + h] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    double2* g = (double2*)(grid + (size_t)row * I);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) g[k] = sz[k];
}

// The device address of g_static_scratch on the current device.  Looked up
// (cudaGetSymbolAddress, with the device current) on every call made
// outside stream capture; a call under capture reuses the address of the
// last uncaptured call on that device and fails if there was none.
mlsdc_status static_scratch(cudaStream_t st, void** out) {
    int dev = 0;
    MLSDC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices)
        return invalid_arg("sh_inverse_static: device ordinal beyond " + std::to_string(kStaticMaxDevices));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t qe = cudaStreamIsCapturing(st, &cs);
    if (qe != cudaSuccess) (void)cudaGetLastError();  // not this call's launch error; treated as capture
    const bool capturing = qe != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!capturing) {
        void* p = nullptr;
        MLSDC_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_ptr[dev] = p;
    } else if (!g_static_ptr[dev]) {
        return invalid_arg("sh_inverse_static: the first call on a device must be made outside stream capture");
    }
    *out = g_static_ptr[dev];
    return MLSDC_OK;
}

}  // namespace
}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status sh_inverse_static(int R, int nlon, int nlat, const double* spec, double* grid, int nf,
                                          void* stream) {
    if (!spec || !grid) return invalid_arg("sh_inverse_static: spec and grid must not be null");
    if (nf < 1 || nf > kMaxFields)
        return invalid_arg("sh_inverse_static: nf must be in [1, " + std::to_string(kMaxFields) + "]");
    if (R < 1) return invalid_arg("sh_inverse_static: R must be >= 1");
    if (nlon < 16 || nlon > 1024 || (nlon & (nlon - 1)) != 0 || nlon < 3 * R + 1)
        return invalid_arg("sh_inverse_static: nlon must be a power of two in [16, 1024] and >= 3R+1");
    if (nlat < 2 || nlat % 2 != 0 || 2 * nlat < 3 * R + 1 || nlat / 2 > kStaticMaxHalfLat)
        return invalid_arg("sh_inverse_static: nlat must be even, >= (3R+1)/2 and <= " +
                           std::to_string(2 * kStaticMaxHalfLat));
    if ((size_t)nf * nlat * (R + 1) > kStaticFourierMax)
        return invalid_arg("sh_inverse_static: nf * nlat * (R+1) exceeds the static scratch of " +
                           std::to_string(kStaticFourierMax) + " complex values");
    MLSDC_ALIGNED("sh_inverse_static", {"spec", spec}, {"grid", grid});
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    mlsdc_status s = static_scratch(st, &base);
    if (s != MLSDC_OK) return s;
    double* lat = (double*)base;
    double2* four = (double2*)((double*)base + kStaticLatDoubles);
    const int J2 = nlat / 2;
    const int nc = nc_of(R);
    k_static_latitudes<<<(J2 + 63) / 64, 64, 0, st>>>(lat, nlat);
    MLSDC_LAUNCHED("k_static_latitudes");
    dim3 gs((J2 + 63) / 64, R + 1, nf);
    k_static_synth<<<gs, 64, 0, st>>>((const double2*)spec, lat, four, R, nlat, nc);
    MLSDC_LAUNCHED("k_static_synth");
    k_static_irfft<<<nf * nlat, 128, sizeof(double2) * (nlon / 2), st>>>(four, grid, R, nlon);
    MLSDC_LAUNCHED("k_static_irfft");
    return MLSDC_OK;
}
