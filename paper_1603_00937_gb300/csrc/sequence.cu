// Pre-determined SP2 branch sequences (Sec. II.C: in the MD run the whole sequence, shared by
// every subgraph, is fixed in advance from a HOMO-LUMO gap estimated at the previous time
// step, so the expansions need no exchange of traces).  Host-only arithmetic; no GPU use.
//
// In the scaled variable x = (e_max - e) / (e_max - e_min) the occupied states lie near 1 and
// the empty ones near 0; the HOMO maps to x_h (largest distance below 1 among occupied
// states), the LUMO to x_l.  The SP2 maps are f1(x) = x^2 and f0(x) = 2x - x^2, so with
// u = 1 - x:  f1: u -> 2u - u^2, f0: u -> u^2.
//
// Gap estimate.  Late in an expansion every eigenvalue but the two interior ones is converged,
// so with e_k = Tr X_k - Tr X_k^2 and d_k = Tr X_k - N_occ,
//     e_k = u_h (1 - u_h) + x_l (1 - x_l),   d_k = x_l - u_h,
// which fixes u_h and x_l at step k; the inverse maps (f1^-1(x) = sqrt(x),
// f0^-1(x) = 1 - sqrt(1 - x)) carry them back to step 0, i.e. to eigenvalues of H.
//
// Sequence.  The two interior eigenvalues are iterated forward with the trace rule applied to
// this two-level system (one occupied level): f1 is taken when |x_h^2 + x_l^2 - 1| is smaller
// than |f0(x_h) + f0(x_l) - 1| (ties take f0), until u_h <= tol and x_l <= tol.
#include <cmath>

#include "gbe_internal.h"

namespace {

// 1 - sqrt(1 - v) without cancellation for small v
double one_minus_sqrt_one_minus(double v) { return v / (1.0 + std::sqrt(1.0 - v)); }

}  // namespace

extern "C" int gbe_sp2_gap_estimate(const gbe_sp2_report* rep, double n_occ, double e_lo, double e_hi, double* homo,
                                    double* lumo) {
    GBE_CHECK_ARG(rep && homo && lumo, "NULL argument");
    GBE_CHECK_ARG(e_lo > 0.0 && e_hi > e_lo && e_hi < 0.5, "need 0 < e_lo < e_hi < 0.5");
    GBE_CHECK_ARG(rep->iters >= 1 && rep->iters <= GBE_SEQ_MAX, "report has no iterations");
    GBE_CHECK_ARG(rep->eps_max > rep->eps_min, "report has no spectral bounds");
    // last step whose idempotency error lies in [e_lo, e_hi]
    int k = -1;
    for (int i = rep->iters; i >= 0; --i) {
        const double e = rep->t1[i] - rep->t2[i];
        if (e >= e_lo && e <= e_hi) { k = i; break; }
    }
    if (k < 0) {
        gbe_set_error("no SP2 step with idempotency error in [%g, %g]", e_lo, e_hi);
        return GBE_EINVAL;
    }
    const double e = rep->t1[k] - rep->t2[k];
    const double d = rep->t1[k] - n_occ;
    // u_h: small root of 2u^2 - (2 - 2d) u - (d - d^2 - e) = 0 (from the two equations above)
    const double b = 2.0 - 2.0 * d;
    const double disc = b * b + 8.0 * (d - d * d - e);
    if (!(disc >= 0.0)) {
        gbe_set_error("traces at step %d are inconsistent with two interior eigenvalues", k);
        return GBE_ENUMERIC;
    }
    double uh = (b - std::sqrt(disc)) / 4.0;
    double xl = uh + d;
    if (!(uh > 0.0 && uh < 0.5 && xl > 0.0 && xl < 0.5)) {
        gbe_set_error("interior eigenvalue estimate out of range at step %d (u_h=%g, x_l=%g)", k, uh, xl);
        return GBE_ENUMERIC;
    }
    for (int j = k - 1; j >= 0; --j) {
        if (rep->seq[j]) {               // x_{j+1} = x_j^2
            uh = one_minus_sqrt_one_minus(uh);
            xl = std::sqrt(xl);
        } else {                         // x_{j+1} = 2 x_j - x_j^2
            uh = std::sqrt(uh);
            xl = one_minus_sqrt_one_minus(xl);
        }
    }
    const double w = rep->eps_max - rep->eps_min;
    *homo = rep->eps_max - (1.0 - uh) * w;
    *lumo = rep->eps_max - xl * w;
    return GBE_OK;
}

extern "C" int gbe_sp2_sequence(double eps_min, double eps_max, double homo, double lumo, double tol, int n_max,
                                uint8_t* seq, int* len) {
    GBE_CHECK_ARG(seq && len, "NULL argument");
    GBE_CHECK_ARG(eps_max > eps_min && eps_min <= homo && homo < lumo && lumo <= eps_max,
                  "need eps_min <= homo < lumo <= eps_max");
    GBE_CHECK_ARG(tol > 0.0 && tol < 0.5 && n_max > 0 && n_max <= GBE_SEQ_MAX, "tol / n_max");
    const double w = eps_max - eps_min;
    double uh = (homo - eps_min) / w;    // 1 - x_h
    double xl = (eps_max - lumo) / w;
    int n = 0;
    while (!(uh <= tol && xl <= tol)) {
        if (n == n_max) {
            *len = n;
            gbe_set_error("gap sequence needs more than n_max=%d steps", n_max);
            return GBE_ENOCONV;
        }
        const double c1 = std::fabs(uh * uh - 2.0 * uh + xl * xl);       // f1: x_h^2 + x_l^2 - 1
        const double c0 = std::fabs(2.0 * xl - xl * xl - uh * uh);       // f0: f0(x_h) + f0(x_l) - 1
        const int b = c1 < c0 ? 1 : 0;
        if (b) { uh = 2.0 * uh - uh * uh; xl = xl * xl; }
        else { uh = uh * uh; xl = 2.0 * xl - xl * xl; }
        seq[n++] = (uint8_t)b;
    }
    *len = n;
    return GBE_OK;
}
