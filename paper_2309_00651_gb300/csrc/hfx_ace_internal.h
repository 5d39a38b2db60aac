// Internal interface between the host library (hfx_api.cu) and the kernels of the rows that
// surround the exchange evaluation: ACE and the overlap screen (hfx_ace.cu), SCDM (hfx_scdm.cu),
// the SIN(R) integrator updates (hfx_sinr.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hfx {
namespace ace {

constexpr int kFormGram = 0;  // C[a][b] = sum_p X[a][p] Y[b][p], split over p, FP64 partials
constexpr int kFormLmul = 1;  // C[m][p] = sum_k T[m][k] Y[k][p] (+ C)

// device error-word bits of a failed factorisation and of a rank-deficient SCDM pick (the
// exchange path uses bits 0 and 1)
constexpr int kErrNotPosDef = 4;
constexpr int kErrRankDeficient = 8;

struct MmArgs {
  const void* x;       // Gram: X [nx][K] FP64 (row stride ldx); lmul: T^T [K][ldx] in the compute type,
                       //   rows 16-byte aligned
  const double* y;     // Gram: Y [ny][K] (row stride ldy); lmul: Y [K][N] (row stride ldy)
  double* out;         // Gram: partials [splits][nx][ny]; lmul: C [nx][N] (row stride ldo)
  long long K;         // contraction length
  long long ldx, ldy, ldo;
  int nx, ny;          // rows of X / T and of Y (Gram)
  long long N;         // lmul: columns
  long long chunk;     // Gram: grid points per split (a multiple of 16)
  int tiles_x, tiles_y, njobs;
  int lower;           // lmul: T is lower triangular (skip k beyond the row tile)
  int accumulate;      // lmul: C += ...
};

// Plan of a split contraction over the grid (Gram form) on `sm_count` SMs.
struct GramPlan {
  int tiles_x, tiles_y, splits, njobs;
  long long chunk;
};
GramPlan gram_plan(int nx, int ny, long long K, int sm_count);
size_t gram_partial_bytes(const GramPlan& p, int nx, int ny);

// Launchers; all asynchronous on `st`, returning the launch error.  `fp32` selects FP32
// products (operands rounded once to FP32), else FP64.
cudaError_t gram(bool fp32, bool absval, const double* x, long long ldx, int nx, const double* y, long long ldy,
                 int ny, long long K, const GramPlan& plan, double* partials, int sm_count, cudaStream_t st);
// v = scale * sum_s partials[s][a][b] (fixed order) to out[a][b] (FP64, row stride ldo) and/or
// to outt[b][a] (FP32 if fp32 else FP64, row stride ldt); either may be NULL
cudaError_t gram_reduce(bool fp32, const double* partials, int splits, int nx, int ny, double scale, double* out,
                        long long ldo, void* outt, long long ldt, cudaStream_t st);
// m <- (m + m^T) / 2 in place (n x n, row stride ld)
cudaError_t symmetrise(double* m, int n, long long ld, cudaStream_t st);
// row stride of a transposed small operand with m columns (16-byte rows)
long long lmul_ldt(bool fp32, int m);
// out[i][p] (+)= sum_k T[i][k] Y[k][p] with T given transposed, tt[k][i] (compute type)
cudaError_t lmul(bool fp32, const void* tt, long long ldt, int m, int k, bool lower, const double* y, long long ldy,
                 long long n, bool accumulate, double* out, long long ldo, int sm_count, cudaStream_t st);
// The same two contractions on the tensor cores (hfx_ace_tc.cu; FP32 contexts): TF32 x 3 split
// products, FP32 accumulation in TMEM.  *_ok tells whether the operands meet their alignment
// and size conditions; a device-side wait that runs out sets the timeout bit of *err.
bool gram_tc_ok(const double* x, long long ldx, const double* y, long long ldy, long long K, const GramPlan& plan);
cudaError_t gram_tc(bool absval, const double* x, long long ldx, int nx, const double* y, long long ldy, int ny,
                    long long K, const GramPlan& plan, double* partials, int* err, int sm_count, cudaStream_t st);
bool lmul_tc_ok(const void* tt, int m, const double* y, double* out);
cudaError_t lmul_tc(const float* tt, long long ldt, int m, int k, const double* y, long long ldy, long long n,
                    bool accumulate, double* out, long long ldo, int* err, int sm_count, cudaStream_t st);
// L (row-major n x n, zeros above the diagonal) with L L^T = -(M + M^T)/2; `work` holds
// n*n + n doubles when the matrix does not fit in shared memory
cudaError_t cholesky_neg_sym(const double* m, long long ldm, int n, double* l, double* work, int* err,
                             int max_smem, cudaStream_t st);
// linvt = (L^-1)^T in the compute type (upper triangular, zeros below), row stride ldt
cudaError_t tri_inverse(bool fp32, const double* l, int n, void* linvt, long long ldt, int max_smem, cudaStream_t st);
// screen compaction: keep i <= j with s[i][j] > cut or i == j, row-major; rowbuf holds n + 1 ints
cudaError_t screen_compact(const double* s, int n, double cut, int32_t* pairs, int64_t* n_pairs, int* rowbuf,
                           cudaStream_t st);

// SCDM: pivots (greedy column-pivoted QR of Psi^T) and qt[i][j] = Q[i][j] in the compute type
// (row stride ldt, the transposed small operand of lmul for Phi = Psi Q); q64 (n x n FP64) may be
// NULL; `scratch` holds scdm_scratch_bytes
size_t scdm_scratch_bytes(bool fp32, int n, long long N, int sm_count);
cudaError_t scdm_pivots_q(bool fp32, const double* psi, long long N, int n, void* scratch, long long* piv, void* qt,
                          long long ldt, double* q64, int* err, int sm_count, cudaStream_t st);

}  // namespace ace
}  // namespace hfx

namespace hfx {
namespace sinr {

constexpr int kMaxChain = 16;  // longest thermostat chain (registers per degree of freedom)

struct SinrArgs {
  double kT, Q1, Q2, gamma;
  int L;
};
struct SyWeights {
  double w[5];
};

// SIN(R) updates A, B, C (hfx_sinr.cu); asynchronous on `st`, returning the launch error
cudaError_t update_n(const SinrArgs& a, long long n_dof, double dt, int n_res, const SyWeights& w, int n_sy,
                     const double* mass, double* V, double* v1, double* v2, cudaStream_t st);
cudaError_t update_v(const SinrArgs& a, long long n_dof, double dt, const double* mass, const double* force,
                     const double* force_extra, double* V, double* v1, cudaStream_t st);
cudaError_t update_x(const SinrArgs& a, long long n_dof, double dt, const double* V, double* X, double* v2,
                     const double* R, cudaStream_t st);

}  // namespace sinr
}  // namespace hfx
