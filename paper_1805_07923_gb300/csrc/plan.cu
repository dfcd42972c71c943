// sh_plan: Gaussian grid, normalised associated Legendre tables and FFT
// twiddles of one truncation (Sec. 3), computed on the host in float64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace mlsdc {

static thread_local std::string g_last_error;

void set_error(const char* where, cudaError_t e) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
}
void set_error_text(const std::string& s) { g_last_error = s; }

mlsdc_status invalid_arg(const std::string& why) {
    g_last_error = why;
    return MLSDC_ERR_INVALID;
}

mlsdc_status check_aligned16(const char* where, std::initializer_list<std::pair<const char*, const void*>> ptrs) {
    for (const auto& pr : ptrs)
        if (((uintptr_t)pr.second & 15u) != 0)
            return invalid_arg(std::string(where) + ": " + pr.first + " is not 16-byte aligned");
    return MLSDC_OK;
}

bool pdl_enabled() {
    // Off by default for every launch: measured inside the step's CUDA graph
    // on GB300, programmatic edges on all launches made the step slower
    // (565 -> 465 steps/s split-BF16, 199 -> 115 float64), although isolated
    // back-to-back launches gained.  The tensor-core analysis alone takes
    // them (PdlScope).
    static const bool on = [] {
        const char* v = std::getenv("MLSDC_PDL");
        return v && v[0] == '1';
    }();
    return on;
}

bool& pdl_scope_flag() {
    thread_local bool on = false;
    return on;
}

void set_carveout_once(const void* kernel) {
    static std::mutex mu;
    static std::vector<const void*> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), kernel) != done.end()) return;
    done.push_back(kernel);
    // a hint: ignore a refusal (the kernel then runs with the driver's choice)
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, kCarveoutPct) != cudaSuccess)
        (void)cudaGetLastError();
}

mlsdc_status raise_smem_limit(const void* fn, size_t bytes) {
    static std::mutex mu;
    if (bytes <= 48 * 1024) return MLSDC_OK;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, fn) == cudaSuccess && (size_t)at.maxDynamicSharedSizeBytes >= bytes)
        return MLSDC_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        set_error("cudaFuncSetAttribute", e);
        return MLSDC_ERR_CUDA;
    }
    return MLSDC_OK;
}

// Gaussian latitudes: roots of the degree-J Legendre polynomial by Newton's
// method, ordered north to south, with weights w = 2 / ((1 - mu^2) P_J'(mu)^2).
static void gaussian_latitudes(int J, std::vector<double>& mu, std::vector<double>& w) {
    mu.assign(J, 0.0);
    w.assign(J, 0.0);
    const double pi = 3.14159265358979323846;
    for (int j = 0; j < (J + 1) / 2; ++j) {
        double x = std::cos(pi * (j + 0.75) / (J + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= J; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = J * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= J; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = J * (x * p1 - p0) / (x * x - 1.0);
        }
        double wj = 2.0 / ((1.0 - x * x) * dp * dp);
        mu[j] = x;
        mu[J - 1 - j] = -x;
        w[j] = wj;
        w[J - 1 - j] = wj;
    }
    if (J % 2 == 1) mu[J / 2] = 0.0;
}

static inline double eps_mn(int m, int n) {
    if (n <= m) return 0.0;
    return std::sqrt((double(n) * n - double(m) * m) / (4.0 * double(n) * n - 1.0));
}

// P^m_n(mu_j) and H^m_n = (1 - mu^2) dP^m_n/dmu for the northern latitudes,
// orthonormal on [-1, 1], no Condon-Shortley phase; |values| < 1e-300 -> 0.
static void legendre_tables(int R, int J2, const std::vector<double>& mu, std::vector<double>& P,
                            std::vector<double>& H) {
    const int nc = nc_of(R);
    P.assign((size_t)nc * J2, 0.0);
    H.assign((size_t)nc * J2, 0.0);
    std::vector<double> col(R + 3);
    for (int j = 0; j < J2; ++j) {
        const double x = mu[j];
        const double s = std::sqrt(1.0 - x * x);
        double pmm = std::sqrt(0.5);
        for (int m = 0; m <= R; ++m) {
            if (m > 0) pmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
            if (std::fabs(pmm) < 1e-300) pmm = 0.0;
            // col[k] = P^m_{m+k}, k = 0 .. R+1-m
            col[0] = pmm;
            double pm1 = 0.0, pn = pmm;
            for (int n = m; n <= R; ++n) {
                double pn1 = (x * pn - eps_mn(m, n) * pm1) / eps_mn(m, n + 1);
                if (std::fabs(pn1) < 1e-300) pn1 = 0.0;
                col[n + 1 - m] = pn1;
                pm1 = pn;
                pn = pn1;
            }
            const int off = moff(R, m);
            for (int n = m; n <= R; ++n) {
                const int k = n - m;
                double pnm1 = (k >= 1) ? col[k - 1] : 0.0;
                double h = -n * eps_mn(m, n + 1) * col[k + 1] + (n + 1.0) * eps_mn(m, n) * pnm1;
                P[(size_t)(off + k) * J2 + j] = col[k];
                H[(size_t)(off + k) * J2 + j] = h;
            }
        }
    }
}

template <class T>
static mlsdc_status dev_alloc(T** ptr, size_t count, int64_t* bytes) {
    cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc", e);
        *ptr = nullptr;
        return MLSDC_ERR_ALLOC;
    }
    *bytes += (int64_t)(count * sizeof(T));
    return MLSDC_OK;
}

static void free_plan(sh_plan_t p) {
    if (!p) return;
    mp_free(p);
    cudaFree(p->d_mu);
    cudaFree(p->d_w);
    cudaFree(p->d_P);
    cudaFree(p->d_H);
    cudaFree(p->d_tw);
    cudaFree(p->d_stab);
    cudaFree(p->d_ndeg);
    cudaFree(p->d_cor);
    cudaFree(p->d_lat);
    cudaFree(p->d_invnn);
    cudaFree(p->d_synth);
    cudaFree(p->d_anal);
    cudaFree(p->d_four_in);
    cudaFree(p->d_four_out);
    delete p;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" const char* mlsdc_status_string(mlsdc_status s) {
    switch (s) {
        case MLSDC_OK: return "ok";
        case MLSDC_ERR_INVALID: return "invalid argument";
        case MLSDC_ERR_CUDA: return "CUDA error";
        case MLSDC_ERR_NONFINITE: return "non-finite state";
        case MLSDC_ERR_TIMEOUT: return "device wait timed out";
        case MLSDC_ERR_ALLOC: return "device allocation failed";
        default: return "unknown status";
    }
}

extern "C" const char* mlsdc_last_error(void) { return g_last_error.c_str(); }

#define TRY(x)                      \
    do {                            \
        mlsdc_status s_ = (x);      \
        if (s_ != MLSDC_OK) {       \
            free_plan(p);           \
            return s_;              \
        }                           \
    } while (0)

extern "C" mlsdc_status sh_plan(int R, int nlon, int nlat, int precision, sh_plan_t* out) {
    return create_plan(R, nlon, nlat, precision, 1, out);
}

extern "C" mlsdc_status sh_plan_batched(int R, int nlon, int nlat, int precision, int max_members,
                                        sh_plan_t* out) {
    return create_plan(R, nlon, nlat, precision, max_members, out);
}

mlsdc_status mlsdc::create_plan(int R, int nlon, int nlat, int precision, int max_members, sh_plan_t* out) {
    if (!out) return MLSDC_ERR_INVALID;
    *out = nullptr;
    if (R < 1 || nlon < 16 || nlon > 1024 || (nlon & (nlon - 1)) != 0 || nlon < 3 * R + 1)
        return MLSDC_ERR_INVALID;
    if (nlat < 2 || nlat % 2 != 0 || 2 * nlat < 3 * R + 1 || nlat / 2 > 1024) return MLSDC_ERR_INVALID;
    if (precision < MLSDC_FP64 || precision > MLSDC_FP32) return MLSDC_ERR_INVALID;
    if (max_members < 1 || max_members > 4096) return MLSDC_ERR_INVALID;

    sh_plan_t p = new sh_plan_s();
    p->max_members = max_members;
    p->R = R;
    p->I = nlon;
    p->J = nlat;
    p->J2 = nlat / 2;
    p->nc = nc_of(R);
    p->precision = precision;
    p->logI = 0;
    while ((1 << p->logI) < nlon) ++p->logI;

    gaussian_latitudes(nlat, p->mu, p->w);
    std::vector<double> P, H;
    legendre_tables(R, p->J2, p->mu, P, H);

    std::vector<double2> tw(nlon / 2);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < nlon / 2; ++k) {
        double ang = 2.0 * pi * k / nlon;
        tw[k] = make_double2(std::cos(ang), -std::sin(ang));
    }
    std::vector<int> ndeg(p->nc);
    for (int m = 0; m <= R; ++m)
        for (int n = m; n <= R; ++n) ndeg[moff(R, m) + n - m] = n;
    // Coriolis factors per coefficient (see coriolis_add): with
    // inv_n = -1/(n(n+1)) (0 for n = 0) and eps zero outside m <= n <= R,
    //   alpha = eps_n - (n-1) eps_n inv_{n-1}   (factor of x_{n-1})
    //   beta  = eps_{n+1} + (n+2) eps_{n+1} inv_{n+1}   (factor of x_{n+1})
    //   gamma = m inv_n
    // (the radius cancels: psi, chi carry a^2 and the H term 1/a^2), padded
    // to four doubles.
    std::vector<double> cor((size_t)4 * p->nc);
    for (int m = 0; m <= R; ++m)
        for (int n = m; n <= R; ++n) {
            auto inv = [](int nn) { return nn > 0 ? -1.0 / (nn * (nn + 1.0)) : 0.0; };
            const double en = eps_mn(m, n), en1 = (n + 1 <= R) ? eps_mn(m, n + 1) : 0.0;
            double* c = &cor[(size_t)4 * (moff(R, m) + n - m)];
            c[0] = en - (n - 1.0) * en * inv(n - 1);
            c[1] = en1 + (n + 2.0) * en1 * inv(n + 1);
            c[2] = m * inv(n);
            c[3] = 0.0;
        }

    // Latitude constants of the grid products and the Fourier weights
    // (Eq. fourier_transform's 1/I and Eq. legendre_transform's w_j), and
    // the inverse Laplacian factors of the Helmholtz step.
    std::vector<double> lat((size_t)4 * nlat), invnn(R + 1);
    for (int j = 0; j < nlat; ++j) {
        const double mu = p->mu[j], w = p->w[j];
        lat[4 * j + 0] = mu;
        lat[4 * j + 1] = 1.0 / (1.0 - mu * mu);
        lat[4 * j + 2] = w / (1.0 - mu * mu) / nlon;
        lat[4 * j + 3] = w / nlon;
    }
    for (int n = 0; n <= R; ++n) invnn[n] = n > 0 ? 1.0 / (n * (n + 1.0)) : 0.0;

    // Legendre work items, largest first so the block scheduler balances them.
    std::vector<Chunk> cs, ca;
    for (int m = 0; m <= R; ++m)
        for (int j0 = 0; j0 < p->J2; j0 += kSynthLat) cs.push_back({m, j0});
    std::stable_sort(cs.begin(), cs.end(), [](const Chunk& a, const Chunk& b) { return a.m < b.m; });
    for (int m = 0; m <= R; ++m)
        for (int k0 = 0; k0 < R + 1 - m; k0 += kAnalRows) ca.push_back({m, k0});
    std::stable_sort(ca.begin(), ca.end(), [R](const Chunk& a, const Chunk& b) {
        int ra = std::min(kAnalRows, R + 1 - a.m - a.start), rb = std::min(kAnalRows, R + 1 - b.m - b.start);
        return ra > rb;
    });
    p->n_synth = (int)cs.size();
    p->n_anal = (int)ca.size();

    const size_t nfour = (size_t)std::max(kMaxFields, 5 * max_members) * nlat * (R + 1);
    TRY(dev_alloc(&p->d_mu, nlat, &p->bytes));
    TRY(dev_alloc(&p->d_w, nlat, &p->bytes));
    TRY(dev_alloc(&p->d_P, P.size(), &p->bytes));
    TRY(dev_alloc(&p->d_H, H.size(), &p->bytes));
    TRY(dev_alloc(&p->d_tw, tw.size(), &p->bytes));
    TRY(dev_alloc(&p->d_ndeg, ndeg.size(), &p->bytes));
    TRY(dev_alloc(&p->d_cor, cor.size(), &p->bytes));
    TRY(dev_alloc(&p->d_lat, lat.size(), &p->bytes));
    TRY(dev_alloc(&p->d_invnn, invnn.size(), &p->bytes));
    TRY(dev_alloc(&p->d_synth, cs.size(), &p->bytes));
    TRY(dev_alloc(&p->d_anal, ca.size(), &p->bytes));
    TRY(dev_alloc(&p->d_four_in, nfour, &p->bytes));
    TRY(dev_alloc(&p->d_four_out, nfour, &p->bytes));

#define H2D(dst, src, n) \
    if (cudaMemcpy(dst, src, (n) * sizeof(*(src)), cudaMemcpyHostToDevice) != cudaSuccess) { \
        set_error("cudaMemcpy", cudaGetLastError()); free_plan(p); return MLSDC_ERR_CUDA; }
    H2D(p->d_mu, p->mu.data(), nlat);
    H2D(p->d_w, p->w.data(), nlat);
    H2D(p->d_P, P.data(), P.size());
    H2D(p->d_H, H.data(), H.size());
    H2D(p->d_tw, tw.data(), tw.size());
    H2D(p->d_ndeg, ndeg.data(), ndeg.size());
    H2D(p->d_cor, cor.data(), cor.size());
    H2D(p->d_lat, lat.data(), lat.size());
    H2D(p->d_invnn, invnn.data(), invnn.size());
    H2D(p->d_synth, cs.data(), cs.size());
    H2D(p->d_anal, ca.data(), ca.size());
#undef H2D
    TRY(f64_prepare(p));
    if (precision != MLSDC_FP64) TRY(mp_init(p));
    *out = p;
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_destroy(sh_plan_t plan) {
    if (!plan) return MLSDC_ERR_INVALID;
    free_plan(plan);
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_grid(sh_plan_t p, double* mu_host, double* w_host) {
    if (!p) return MLSDC_ERR_INVALID;
    if (mu_host) std::memcpy(mu_host, p->mu.data(), sizeof(double) * p->J);
    if (w_host) std::memcpy(w_host, p->w.data(), sizeof(double) * p->J);
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_plan_device_bytes(sh_plan_t p, int64_t* bytes) {
    if (!p || !bytes) return MLSDC_ERR_INVALID;
    *bytes = p->bytes + p->mp.tc_bytes;
    return MLSDC_OK;
}

namespace mlsdc {
mlsdc_status tc_error(sh_plan_t p, int* code);
mlsdc_status mp_error(sh_plan_t p, int* code);
}

extern "C" mlsdc_status sh_plan_device_error(sh_plan_t p, int* code) {
    if (!p || !code) return MLSDC_ERR_INVALID;
    *code = 0;
    if (p->precision == MLSDC_FP64) return MLSDC_OK;
    MLSDC_CUDA(cudaDeviceSynchronize());
    int c_mp = 0, c_tc = 0;
    mlsdc_status s = mlsdc::mp_error(p, &c_mp);
    if (s == MLSDC_OK && (p->precision == MLSDC_TF32 || p->precision == MLSDC_BF16X3)) s = mlsdc::tc_error(p, &c_tc);
    *code = c_tc ? c_tc : c_mp;
    return s;
}
