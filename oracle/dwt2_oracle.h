/* dwt2_oracle.h -- CPU oracle for the 2-D discrete wavelet transform by lifting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path includes, links or calls this
 * code: only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares
 * no header, table or helper with the CUDA library.
 *
 * Conventions (the paper's, Sec. 2):
 *   - image row-major, H rows x W columns; "horizontal" = along a row = the m / z_m axis,
 *     "vertical" = along a column = the n / z_n axis;
 *   - polyphase quad at (n, m): LL = x[2n][2m], HL = x[2n][2m+1], LH = x[2n+1][2m],
 *     HH = x[2n+1][2m+1], i.e. the vector order [LL, HL, LH, HH] of Eq. 3 / Eq. 5;
 *   - one level maps an h x w plane to LL ceil(h/2) x ceil(w/2), HL ceil(h/2) x floor(w/2),
 *     LH floor(h/2) x ceil(w/2), HH floor(h/2) x floor(w/2);
 *   - multi-level (Mallat) recursion on LL; band list order LL_J, then for j = J..1:
 *     HL_j, LH_j, HH_j, each band stored densely (row stride = its width);
 *   - boundaries: whole-sample symmetric extension x[-k] = x[k], x[N-1+k] = x[N-1-k];
 *     an axis of length 1 passes through unchanged.
 *
 * Wavelets: ORC_CDF53_INT (reversible integer CDF 5/3, exact int64, floor division),
 *           ORC_CDF53     (CDF 5/3 in fp64), ORC_CDF97 (CDF 9/7 in fp64),
 *           ORC_DD97, ORC_DD137 (Deslauriers-Dubuc 9/7 and 13/7 in fp64: four-tap predict,
 *           two- or four-tap update, no scaling).  The Deslauriers-Dubuc wavelets have the
 *           forward and inverse transforms of the separable and non-separable schemes; the
 *           adjoints, the adapted scheme and the step-by-step entry points are for the CDF
 *           wavelets only.
 * All functions return 0 on success and a negative value on invalid arguments.
 */
#ifndef DWT2_ORACLE_H
#define DWT2_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_CDF53_INT = 0, ORC_CDF53 = 1, ORC_CDF97 = 2, ORC_DD97 = 3, ORC_DD137 = 4 };

/* Schemes: how one level is evaluated.
 *   ORC_SEP_EQ3      separable lifting, steps P_h, P_v, U_h, U_v per lifting pair (Eq. 3)
 *   ORC_SEP_ROWS     the whole 1-D transform along rows, then along columns
 *   ORC_SEP_COLS     the whole 1-D transform along columns, then along rows
 *   ORC_NONSEP_EQ5   fused spatial predict / spatial update steps (Eq. 5)
 *   ORC_ADAPTED      the adapted non-separable scheme (Sec. 3, Fig. 3): P = P0 + P1 and
 *                    U = U0 + U1 with P0, U0 the constant monomials; each spatial step of Eq. 5
 *                    becomes a local step with the constants (no neighbouring quad is read)
 *                    followed by the fused step with P1, U1.  Float wavelets, forward only.
 * For the integer wavelet only ORC_SEP_EQ3 and ORC_NONSEP_EQ5 are the contract (they agree
 * bit for bit); the other orders round differently. */
enum { ORC_SEP_EQ3 = 0, ORC_SEP_ROWS = 1, ORC_SEP_COLS = 2, ORC_NONSEP_EQ5 = 3, ORC_ADAPTED = 4 };

/* Boundary evaluation for the separable schemes:
 *   0: single whole-sample reflection inside each lifting step (x[-1] = x[1], x[N] = x[N-2]);
 *   1: the signal is first extended by repeated whole-sample reflection (period 2N-2) and
 *      lifted with no boundary rule at all, then cropped.  Both must agree. */

/* Threads for the line loops of the separable steps (default 1, the sequential oracle).  More
 * threads share out the independent lines of each 1-D step; every value is computed the same
 * way, so results are bit-identical for any count.  Returns the count in effect. */
int orc_set_threads(int n);

int orc_max_levels(int H, int W);
/* number of elements of the concatenated band list for (H, W, levels) */
int64_t orc_coeff_count(int H, int W, int levels);

/* Forward transform.  img: H*W values (int64 for ORC_CDF53_INT, double otherwise).
 * out: orc_coeff_count values of the same type, band list order. */
int orc_forward(const void* img, int H, int W, int wavelet, int levels, int scheme,
                int extension_form, void* out);
/* Inverse transform: band list -> H*W image. */
int orc_inverse(const void* coeffs, int H, int W, int wavelet, int levels, int scheme,
                void* img);
/* Transpose of the forward transform (float wavelets): band-list gradient -> image gradient. */
int orc_forward_adjoint(const double* g_coeffs, int H, int W, int wavelet, int levels,
                        double* g_img);
/* Transpose of the inverse transform (float wavelets): image gradient -> band-list gradient. */
int orc_inverse_adjoint(const double* g_img, int H, int W, int wavelet, int levels,
                        double* g_coeffs);

/* The first nsteps fused steps of Eq. 5 (spatial predict, spatial update, predict, ...) of one
 * level, without the 9/7 scaling; out receives the four polyphase components a (LL), b (HL),
 * c (LH), e (HH) densely, in that order.  Used to check which components each step writes. */
int orc_nonsep_steps(const double* img, int H, int W, int wavelet, int nsteps, double* out);

/* The same for the adapted scheme: steps in order local predict (P0), fused predict (P1),
 * local update (U0), fused update (U1), ... of one level, without the 9/7 scaling. */
int orc_adapted_steps(const double* img, int H, int W, int wavelet, int nsteps, double* out);
/* Applies adapted steps k0 .. k1-1 (numbered as above) in place to polyphase components given
 * densely in abce (a, b, c, e of an H x W level, the layout orc_adapted_steps writes). */
int orc_adapted_apply(double* abce, int H, int W, int wavelet, int k0, int k1);

#ifdef __cplusplus
}
#endif
#endif
