// Float64 spherical-harmonic transforms (Sec. 3, Eqs. spectral_to_physical_space,
// fourier_transform, legendre_transform) and the float64 instantiation of
// the explicit right-hand side F_E (rhs_kernels.cuh).  Also the stage timing
// entry point used for roofline reporting.
#include <cmath>

#include "complex.cuh"
#include "internal.h"
#include "rhs_kernels.cuh"

namespace mlsdc {

// ---------------------------------------------------------------------------
// Scalar transforms (sh_inverse / sh_forward).
__global__ void __launch_bounds__(32) k_synth_scalar_f64(const double2* __restrict__ spec,
                                                         const double* __restrict__ P,
                                                         const Chunk* __restrict__ chunks, int R,
                                                         int J2, int nc, double2* __restrict__ four) {
    extern __shared__ double2 sc[];
    const int fld = blockIdx.y;
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    for (int k = threadIdx.x; k < nm; k += blockDim.x) sc[k] = spec[(size_t)fld * nc + off + k];
    __syncthreads();
    const int j = ch.start + threadIdx.x;
    if (j >= J2) return;
    double2 e{0, 0}, o{0, 0};
    const double* Pm = P + (size_t)off * J2 + j;
    int k = 0;
    for (; k + 1 < nm; k += 2) {
        cfma(e, Pm[(size_t)k * J2], sc[k]);
        cfma(o, Pm[(size_t)(k + 1) * J2], sc[k + 1]);
    }
    if (k < nm) cfma(e, Pm[(size_t)k * J2], sc[k]);
    const int J = 2 * J2;
    const size_t base = (size_t)fld * J * (R + 1);
    four[base + (size_t)j * (R + 1) + m] = cadd(e, o);
    four[base + (size_t)(J - 1 - j) * (R + 1) + m] = csub(e, o);
}

// Inverse real DFT of one row per block: coefficients m <= R -> I grid values.
__global__ void __launch_bounds__(128) k_fft_inv_rows_f64(const double2* __restrict__ four,
                                                          double* __restrict__ grid,
                                                          const double2* __restrict__ tw, int R, int I,
                                                          int logI) {
    extern __shared__ double2 sx[];
    const int row = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    const double2* F = four + (size_t)row * (R + 1);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) sx[bitrev(k, logH)] = irfft_pack(F, k, R, Hn, tw);
    __syncthreads();
    fft_dit(sx, 1, Hn, logH, tw, true);
    double2* g = (double2*)(grid + (size_t)row * I);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) g[k] = sx[k];
}

// Forward real DFT of one row per block, coefficients m <= R scaled by w_j / I.
__global__ void __launch_bounds__(128) k_fft_fwd_rows_f64(const double* __restrict__ grid,
                                                          double2* __restrict__ four,
                                                          const double* __restrict__ w,
                                                          const double2* __restrict__ tw, int R, int I,
                                                          int logI, int J) {
    extern __shared__ double2 sx[];
    const int row = blockIdx.x;
    const int Hn = I >> 1, logH = logI - 1;
    const double2* g = (const double2*)(grid + (size_t)row * I);
    for (int k = threadIdx.x; k < Hn; k += blockDim.x) sx[bitrev(k, logH)] = g[k];
    __syncthreads();
    fft_dit(sx, 1, Hn, logH, tw, false);
    const double s = w[row % J] / I;
    for (int m = threadIdx.x; m <= R; m += blockDim.x)
        four[(size_t)row * (R + 1) + m] = cscale(rfft_unpack(sx, m, Hn, tw), s);
}

__global__ void __launch_bounds__(32) k_anal_scalar_f64(const double2* __restrict__ four,
                                                        const double* __restrict__ P,
                                                        const Chunk* __restrict__ chunks, int R, int J2,
                                                        int nc, double2* __restrict__ spec) {
    __shared__ double2 sG[32][2];
    __shared__ double sP[32][33];
    const int fld = blockIdx.y;
    const Chunk ch = chunks[blockIdx.x];
    const int m = ch.m;
    const int nm = R + 1 - m;
    const int off = m * (R + 1) - m * (m - 1) / 2;
    const int k0 = ch.start;
    const int lane = threadIdx.x;
    const int par = (k0 + lane) & 1;
    const int J = 2 * J2;
    const double2* F = four + (size_t)fld * J * (R + 1);
    const int rows = min(32, nm - k0);
    double2 acc{0, 0};
    for (int jt = 0; jt < J2; jt += 32) {
        const int nl = min(32, J2 - jt);
        if (lane < nl) {
            const double2 gN = F[(size_t)(jt + lane) * (R + 1) + m];
            const double2 gS = F[(size_t)(J - 1 - jt - lane) * (R + 1) + m];
            sG[lane][0] = cadd(gN, gS);
            sG[lane][1] = csub(gN, gS);
        }
        for (int r = 0; r < rows; ++r)
            if (lane < nl) sP[r][lane] = P[(size_t)(off + k0 + r) * J2 + jt + lane];
        __syncwarp();
        if (lane < rows)
            for (int jj = 0; jj < nl; ++jj) cfma(acc, sP[lane][jj], sG[jj][par]);
        __syncwarp();
    }
    if (lane >= rows) return;
    if (m == 0) acc.y = 0.0;
    spec[(size_t)fld * nc + off + k0 + lane] = acc;
}

mlsdc_status f64_prepare(sh_plan_t p) {
    mlsdc_status s;
    MLSDC_CUDA(cudaMalloc((void**)&p->d_stab, (size_t)(p->I / 2) * sizeof(double2)));
    p->bytes += (int64_t)(p->I / 2) * sizeof(double2);
    k_stage_twiddles<double2><<<1, 256>>>(p->d_stab, p->d_tw, p->I / 2, p->logI - 1, p->I);
    MLSDC_LAUNCHED("k_stage_twiddles");
    if ((s = raise_smem_limit((const void*)k_grid_rhs<double, 1>, grid_smem<double>(p->I))) != MLSDC_OK) return s;
    if ((s = raise_smem_limit((const void*)k_synth_rhs<double, false>, synth_smem<double>(p->R))) != MLSDC_OK) return s;
    return MLSDC_OK;
}

mlsdc_status rhs_explicit_f64(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                              cudaStream_t st, int64_t* launches, int stage, RhsBatch b) {
    const int R = p->R;
    if (b.members < 1 || b.members > p->max_members) return MLSDC_ERR_INVALID;
    const size_t fs = (size_t)p->J * (R + 1);
    const MemberStrides ms{b.state_ms, 4 * fs, 5 * fs, b.fe_ms};
    const FourStride fo = four_out_layout(p->J, R, false);  // float64 path: m-contiguous
    if (stage == 0 || stage < 0) {
        MLSDC_LAUNCH("k_synth_rhs<double>",
                     launch_b(Body::SynthF64, 0, 0, k_synth_rhs<double, false>, dim3(p->n_synth, b.members), dim3(32 * kSynthWarps),
                              synth_smem<double>(R), st, SynMaps{}, (int*)nullptr, (const double2*)state,
                              (const double*)p->d_P,
                              (const double*)p->d_H, (const double*)p->d_invnn, (const Chunk*)p->d_synth, R, p->J2,
                              p->nc, -prm->a * prm->a, 1.0 / prm->a, p->d_four_in, ms));
    }
    if (stage == 1 || stage < 0) {
        MLSDC_LAUNCH("k_grid_rhs<double>",
                     launch_b(Body::GridF64x1, 0, 0, k_grid_rhs<double, 1>, dim3(p->J, b.members), dim3(256), grid_smem<double>(p->I),
                              st, (const double2*)p->d_four_in, p->d_four_out, (const double*)p->d_lat,
                              (const double2*)p->d_tw, (const double2*)p->d_stab, R, p->I, p->logI, p->J, 2.0 * prm->omega, ms,
                              fo));
    }
    if (stage == 2 || stage < 0) {
        MLSDC_LAUNCH("k_anal_rhs<double>",
                     launch_b(Body::AnalF64, 0, anal_smem_bytes<double>(), k_anal_rhs<double>, dim3(p->n_anal, b.members), dim3(32 * anal_warps(p->J2)), 0, st,
                              (const double2*)p->d_four_out, (const double*)p->d_P, (const double*)p->d_H,
                              (const Chunk*)p->d_anal, R, p->J2, p->nc, 1.0 / prm->a, (double2*)FE,
                              (const double2*)state, 0.0, (const double*)p->d_cor, ms, fo));
    }
    if (launches) *launches += stage < 0 ? 3 : 1;
    return MLSDC_OK;
}

}  // namespace mlsdc

using namespace mlsdc;

extern "C" mlsdc_status sh_inverse(sh_plan_t p, const double* spec, double* grid, int nf, void* stream) {
    if (!p || !spec || !grid || nf < 1 || nf > kMaxFields) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("sh_inverse", {"spec", spec}, {"grid", grid});
    cudaStream_t st = (cudaStream_t)stream;
    const int R = p->R;
    dim3 gs(p->n_synth, nf);
    k_synth_scalar_f64<<<gs, 32, sizeof(double2) * (R + 1), st>>>((const double2*)spec, p->d_P, p->d_synth, R,
                                                                  p->J2, p->nc, p->d_four_in);
    MLSDC_LAUNCHED("k_synth_scalar_f64");
    const int rows = nf * p->J;
    k_fft_inv_rows_f64<<<rows, 128, sizeof(double2) * (p->I / 2), st>>>(p->d_four_in, grid, p->d_tw, R, p->I,
                                                                        p->logI);
    MLSDC_LAUNCHED("k_fft_inv_rows_f64");
    return MLSDC_OK;
}

extern "C" mlsdc_status sh_forward(sh_plan_t p, const double* grid, double* spec, int nf, void* stream) {
    if (!p || !spec || !grid || nf < 1 || nf > kMaxFields) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("sh_forward", {"grid", grid}, {"spec", spec});
    cudaStream_t st = (cudaStream_t)stream;
    const int R = p->R;
    const int rows = nf * p->J;
    k_fft_fwd_rows_f64<<<rows, 128, sizeof(double2) * (p->I / 2), st>>>(grid, p->d_four_out, p->d_w, p->d_tw, R,
                                                                        p->I, p->logI, p->J);
    MLSDC_LAUNCHED("k_fft_fwd_rows_f64");
    dim3 ga(p->n_anal, nf);
    k_anal_scalar_f64<<<ga, 32, 0, st>>>(p->d_four_out, p->d_P, p->d_anal, R, p->J2, p->nc, (double2*)spec);
    MLSDC_LAUNCHED("k_anal_scalar_f64");
    return MLSDC_OK;
}

extern "C" mlsdc_status swe_explicit_rhs(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                                         void* stream) {
    if (!p || !prm || !state || !FE || state == FE) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_explicit_rhs", {"state", state}, {"FE", FE});
    cudaStream_t st = (cudaStream_t)stream;
    if (p->precision == MLSDC_FP64) return rhs_explicit_f64(p, prm, state, FE, st, nullptr, -1);
    return rhs_explicit_mp(p, prm, state, FE, st, nullptr, -1);
}

extern "C" mlsdc_status swe_explicit_rhs_batched(sh_plan_t p, const swe_params* prm, const double* states, double* FE,
                                                 int members, void* stream) {
    if (!p || !prm || !states || !FE || states == FE || members < 1 || members > p->max_members)
        return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("swe_explicit_rhs_batched", {"states", states}, {"FE", FE});
    RhsBatch b;
    b.members = members;
    b.state_ms = b.fe_ms = (size_t)3 * p->nc;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->precision == MLSDC_FP64) return rhs_explicit_f64(p, prm, states, FE, st, nullptr, -1, b);
    return rhs_explicit_mp(p, prm, states, FE, st, nullptr, -1, b);
}

extern "C" mlsdc_status mlsdc_profile_rhs(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                                          int reps, float* ms_host, void* stream) {
    return mlsdc_profile_rhs_batched(p, prm, state, FE, 1, reps, ms_host, stream);
}

extern "C" mlsdc_status mlsdc_profile_rhs_batched(sh_plan_t p, const swe_params* prm, const double* state, double* FE,
                                                  int members, int reps, float* ms_host, void* stream) {
    if (!p || !prm || !state || !FE || state == FE || reps < 1 || !ms_host) return MLSDC_ERR_INVALID;
    MLSDC_ALIGNED("mlsdc_profile_rhs", {"state", state}, {"FE", FE});
    if (members < 1 || members > p->max_members) return MLSDC_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    RhsBatch b;
    b.members = members;
    b.state_ms = b.fe_ms = (size_t)3 * p->nc;
    auto run = [&](int stage, cudaStream_t s) {
        return p->precision == MLSDC_FP64 ? rhs_explicit_f64(p, prm, state, FE, s, nullptr, stage, b)
                                          : rhs_explicit_mp(p, prm, state, FE, s, nullptr, stage, b);
    };
    // one full evaluation first so every stage reads valid inputs
    mlsdc_status s = run(-1, st);
    if (s != MLSDC_OK) return s;
    for (int stage = 0; stage < 3 && s == MLSDC_OK; ++stage)
        s = time_in_graph(st, reps, &ms_host[stage], [&](cudaStream_t cs) { return run(stage, cs); });
    return s;
}
