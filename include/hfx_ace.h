/* hfx_ace.h -- C ABI of the adaptively compressed exchange (ACE) operator and of the
 * overlap screen of the pair list, on the same context as the exchange evaluation (hfx.h).
 *
 * ACE (Sec. 2.1, Eq. vx_ace and the definitions of P, W, L and M that follow it), for real
 * orbitals on the context's grid with the grid inner product <f|g> = (Omega/N) sum_p f g:
 *
 *   W_l   = V_x psi_l                     (what hfx_apply returns in `vxphi`)
 *   M_kl  = <psi_k | W_l>
 *   L L^T = -(M + M^T)/2                  (Cholesky; M is symmetric for the full pair list,
 *                                          its symmetric part is taken for any list)
 *   P     = W L^-T                        (rows: P_k = sum_l (L^-1)_kl W_l)
 *   V_x^ACE chi = - sum_k P_k <P_k | chi>
 *
 * Screen (Sec. 2.1, the overlap cut of the localised-orbital variant):
 *   s_ij = (Omega/N) sum_p |phi_i(r_p)| |phi_j(r_p)|; pair i <= j is kept when s_ij > cut,
 *   diagonal pairs always; pairs come out in row-major (i, then j) order.
 *
 * Layout: every grid function is a row of N = n1 n2 n3 FP64 values (z fastest), functions
 * stacked as [count][n1][n2][n3]; small matrices are row-major FP64.  All pointers are
 * device pointers owned by the caller, as is the workspace (hfx_ace_workspace_bytes).
 *
 * Arithmetic follows the context's precision: HFX_PREC_FP64 contracts in FP64; HFX_PREC_FP32
 * rounds each operand to FP32 (nearest) for the products and sums in FP32 over runs of at
 * most 256 terms, FP64 beyond; the Cholesky factorisation and the triangular inverse are FP64
 * in both.  Calls are asynchronous on `cuda_stream`; argument errors return on the host before
 * any launch.  A pivot <= 0 in the factorisation sets the context's device error word
 * (hfx_sync_status then returns HFX_ERR_NOT_POSITIVE_DEFINITE) and leaves L and P undefined.
 */
#ifndef HFX_ACE_H
#define HFX_ACE_H

#include "hfx.h"

#ifdef __cplusplus
extern "C" {
#endif

/* hfx_ace_workspace_bytes -- device workspace that hfx_ace_build (n_psi = 0), hfx_ace_apply
 * and hfx_screen_pairs need for n_orb orbitals and n_psi functions: the split-contraction
 * partial sums plus the small matrices.  0 when the sizes are invalid.  (Library plumbing: the
 * paper has no counterpart.) */
size_t hfx_ace_workspace_bytes(const hfx_ctx* c, int32_t n_orb, int32_t n_psi);

/* hfx_ace_build -- ACE construction from the occupied orbitals and their exchange action
 * (Sec. 2.1, Eq. vx_ace and the definitions of M, L and P after it).
 *   orbitals : [n_orb][N] FP64, read only (psi).
 *   w        : [n_orb][N] FP64, read only (W = V_x psi, e.g. the output of hfx_apply).
 *   m        : [n_orb][n_orb] FP64 out, M_kl = <psi_k|W_l> as defined (not symmetrised); may be
 *              NULL (then held in the workspace).
 *   l        : [n_orb][n_orb] FP64 out, the lower Cholesky factor of -(M + M^T)/2 with zeros
 *              above the diagonal; may be NULL.
 *   p        : [n_orb][N] FP64 out, P = W L^-T stored as rows; must not overlap the inputs.
 * HFX_ERR_INVALID_ARG for NULL inputs or p, n_orb < 1, misaligned (8-byte) pointers;
 * HFX_ERR_OOM when the workspace is short. */
hfx_status hfx_ace_build(hfx_ctx* c, const double* orbitals, const double* w, int32_t n_orb, double* m,
                         double* l, double* p, void* workspace, size_t workspace_bytes, void* cuda_stream);

/* hfx_ace_apply -- out_i = V_x^ACE psi_i = - sum_k P_k <P_k|psi_i> for i < n_psi (Sec. 2.1,
 * Eq. vx_ace: the compressed operator applied on the inner steps).
 *   p   : [n_orb][N] FP64 (from hfx_ace_build), read only.
 *   psi : [n_psi][N] FP64, read only.
 *   out : [n_psi][N] FP64; overwritten, or added to with HFX_ACCUMULATE in `flags`; must not
 *         overlap p or psi. */
hfx_status hfx_ace_apply(hfx_ctx* c, const double* p, int32_t n_orb, const double* psi, int32_t n_psi,
                         uint32_t flags, double* out, void* workspace, size_t workspace_bytes,
                         void* cuda_stream);

/* hfx_screen_pairs -- the overlap screen of the pair list (Sec. 2.1, the overlap cut of the
 * localised-orbital variant, s-MTACE).
 *   orbitals : [n_orb][N] FP64, read only.
 *   cut      : keep i < j when s_ij > cut (finite, >= 0).
 *   s        : [n_orb][n_orb] FP64 out (symmetric), or NULL.
 *   pairs    : int32 [n_orb (n_orb + 1) / 2][2] out (capacity of the full list); the first
 *              *n_pairs rows hold the kept pairs, row-major.
 *   n_pairs  : device int64 out, the number of kept pairs (>= n_orb). */
hfx_status hfx_screen_pairs(hfx_ctx* c, const double* orbitals, int32_t n_orb, double cut, double* s,
                            int32_t* pairs, int64_t* n_pairs, void* workspace, size_t workspace_bytes,
                            void* cuda_stream);

/* hfx_scdm_workspace_bytes -- device workspace of hfx_scdm_localise for n_orb orbitals
 * (residual norms, per-block maxima, Q in the compute type; FP32 contexts also an FP32 copy of
 * the orbitals).  0 when the sizes are invalid.  (Library plumbing: the paper has no
 * counterpart.) */
size_t hfx_scdm_workspace_bytes(const hfx_ctx* c, int32_t n_orb);

/* hfx_scdm_localise -- SCDM localisation (the selected-columns-of-the-density-matrix method the
 * paper's localised-orbital variant uses, Sec. 2.1): a column-pivoted QR factorisation of Psi^T
 * (greedy: at step j the grid point whose orbital-value column has the largest residual norm
 * after removing q_0..q_{j-1}, lowest index on a tie) picks n_orb grid points, q_j is the unit
 * residual of the picked column, and the localised orthonormal orbitals are Phi = Psi Q
 * (Phi_j = sum_i Q[i][j] psi_i).
 *   orbitals : [n_orb][N] FP64, read only, 1 <= n_orb <= min(N, 768).
 *   pivots   : device int64 [n_orb] out, the picked grid points in order (flat index, z fastest).
 *   q        : [n_orb][n_orb] FP64 out (columns q_j), or NULL.
 *   phi_loc  : [n_orb][N] FP64 out; must not overlap the orbitals.
 * FP32 contexts round the orbitals once to FP32 for the residual updates (residual norms in
 * FP64), so a pick may differ from the FP64 one where two residual norms agree to ~1e-6;
 * HFX_ERR_RANK_DEFICIENT (via hfx_sync_status) when the orbitals span fewer than n_orb grid
 * columns. */
hfx_status hfx_scdm_localise(hfx_ctx* c, const double* orbitals, int32_t n_orb, int64_t* pivots, double* q,
                             double* phi_loc, void* workspace, size_t workspace_bytes, void* cuda_stream);

/* hfx_ace_profile_read -- (measurement; the paper has no counterpart) per-kernel device time of
 * the calls above while hfx_profile_enable
 * is on (CUDA events around each launch on the call's stream): summed milliseconds and launch
 * counts since the last read, then reset; index 0 the split grid contractions (M, <psi|P>, s),
 * 1 the left multiplies (P, V_x^ACE psi, Phi = Psi Q), 2 the other steps (partial-sum
 * reduction, Cholesky factorisation, triangular inverse, pair compaction, the SCDM picks and
 * residual updates).  Not for use inside stream capture. */
hfx_status hfx_ace_profile_read(hfx_ctx* c, double ms[3], int64_t launches[3]);

#ifdef __cplusplus
}
#endif

#endif /* HFX_ACE_H */
