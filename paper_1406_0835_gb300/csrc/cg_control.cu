// Device-side control of the CG minimisation (the paper names nonlinear CG
// without details; this is the library's reading, identical to the oracle's):
// Polak-Ribiere+ directions projected orthogonal to phi, restart along -g when
// not descending, norm-preserving rotation phi cos(theta) + dhat sin(theta),
// line search on dE/dtheta (secant, regula falsi once bracketed) until
// |dE/dtheta| <= ls_tol |dE/dtheta(0)| at a point below the sufficient-decrease
// line E(0) + 1e-4 theta dE/dtheta(0) (+ a rounding allowance), stop at
// ||g|| < gtol.
//
// Each controller is one thread: it reads the sums the reductions wrote into
// the CgState, updates the scalars the vector kernels read, and sets the
// conditional handles that drive the graph's WHILE loops.
#include <math.h>

#include "kernels.h"

namespace ofdft {

namespace {

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, unsigned v)
{
    if (use) cudaGraphSetConditional(h, v);
}

// Electronic energy (E_H + E_loc + F_s + F_xc) from the evaluation sums.
__device__ __forceinline__ double e_elec(const CgState *s, const double *ev)
{
    return ev[0] + ev[1] + s->dV * (ev[s->eoff] + ev[s->eoff + 2]);
}

__global__ void k_ctl_norm(CgState *s)
{
    double ss = s->rn[0] * s->dV;
    if (!(ss > 0.0) || !isfinite(ss)) {
        s->scale = 1.0;
        s->status = OFDFT_ENUMERIC;
        s->done = 1;
        return;
    }
    s->scale = sqrt(s->Ne / ss);
}

__global__ void k_ctl_init(CgState *s)
{
    s->mu = s->ev[15] / s->ev[16];
    for (int k = 0; k < 18; ++k) s->ev_acc[k] = s->ev[k];
    s->nevals = 1;
    s->it = 0;
    s->have_prev = 0;
    s->beta = 0.0;
    s->theta_prev = s->theta0;
    if (s->status != OFDFT_ENUMERIC) {
        s->done = 0;
        s->status = OFDFT_ENOCONV;
    }
    s->best_g = INFINITY;
    s->best_it = 0;
    s->accepted = 0;
    s->gg = 0.0;
    s->nouter = 0;
}

__global__ void k_ctl_grad(CgState *s, int first, cudaGraphConditionalHandle outer, int use)
{
    if (first) {
        s->gg = s->rg[0];
        s->have_prev = 0;
        s->beta = 0.0;
    } else if (s->accepted) {
        s->ggprev = s->gg;
        s->gg = s->rg[0];
        double b = (s->gg - s->rg[1]) / s->ggprev;
        s->beta = b > 0.0 ? b : 0.0;
        s->have_prev = 1;
        s->it += 1;
    }
    s->gnorm = sqrt(s->dV * s->gg);
    if (!isfinite(s->gnorm) || !isfinite(s->mu)) {
        s->status = OFDFT_ENUMERIC;
        s->done = 1;
    }
    if (!s->done) {
        if (s->gnorm < s->gtol) {
            s->status = OFDFT_OK;
            s->done = 1;
        } else if (s->it >= s->maxit) {
            s->done = 1;
        } else if (s->stagnate && s->gnorm < s->switch_g) {
            s->status = kCgStagnated;
            s->done = 1;
        } else if (s->stagnate) {
            if (s->gnorm < 0.9 * s->best_g) {
                s->best_g = s->gnorm;
                s->best_it = s->it;
            } else if (s->it - s->best_it >= s->stagnate) {
                s->status = kCgStagnated;
                s->done = 1;
            }
        }
    }
    set_cond(outer, use, s->done ? 0u : 1u);
}

__global__ void k_ctl_dir(CgState *s)
{
    const double sphd = s->rd[0], sdd = s->rd[1], sdg = s->rd[2], spp = s->rd[3], spg = s->rd[4];
    double c1 = sphd / spp;
    double dg = sdg - c1 * spg;
    double dd = sdd - 2.0 * c1 * sphd + c1 * c1 * spp;
    int restart = dg >= 0.0;
    s->c1 = c1;
    s->c2 = restart ? sqrt(spp / s->gg) : sqrt(spp / dd);
    s->restart = restart;
    s->c12r[0] = s->c1;
    s->c12r[1] = s->c2;
    s->c12r[2] = restart ? 1.0 : 0.0;
    s->nouter += 1;
}

__global__ void k_ctl_dhat(CgState *s, cudaGraphConditionalHandle ls, int use)
{
    s->D0 = s->dV * s->rh[0];
    s->lo = 0.0;
    s->Dlo = s->D0;
    s->hi = -1.0;
    s->Dhi = 0.0;
    s->pa = 0.0;
    s->Da = s->D0;
    s->E0 = e_elec(s, s->ev_acc);
    s->hi_nod = 0;
    s->th = s->theta_prev;
    s->nls = 0;
    s->fallback = 0;
    s->accepted = 0;
    s->cs[0] = cos(s->th);
    s->cs[1] = sin(s->th);
    s->csf[0] = (float)s->cs[0];
    s->csf[1] = (float)s->cs[1];
    s->ls_active = 1;
    set_cond(ls, use, 1u);
}

__global__ void k_ctl_ls(CgState *s, cudaGraphConditionalHandle ls, int use)
{
    s->nls += 1;
    s->nevals += 1;
    const double D = s->dV * s->ev[17];
    bool accept = false, failed = false;
    // energy safeguard: a trial above the sufficient-decrease line bounds the
    // step from above whatever the sign of D there
    bool up = false;
    if (s->e_tol > 0.0)
        up = e_elec(s, s->ev) > s->E0 + 1e-4 * s->th * s->D0 + s->e_tol * fabs(s->E0);
    if (s->fallback) {
        accept = true;
    } else if (!up && fabs(D) <= s->ls_tol * fabs(s->D0)) {
        accept = true;
    } else {
        if (up) {
            s->hi = s->th;
            s->Dhi = D;
            s->hi_nod = D > 0.0 ? 0 : 1;
        } else if (D < 0.0) {
            s->lo = s->th;
            s->Dlo = D;
        } else {
            s->hi = s->th;
            s->Dhi = D;
            s->hi_nod = 0;
        }
        if (s->nls >= s->max_ls) {
            if (s->lo > 0.0) {          // one more evaluation at the best descent point
                s->fallback = 1;
                s->th = s->lo;
            } else {
                failed = true;
            }
        } else {
            double nxt;
            if (s->hi < 0.0) {
                nxt = 4.0 * s->th;
                if (D > s->Da) {
                    double sec = s->th - D * (s->th - s->pa) / (D - s->Da);
                    nxt = sec < 4.0 * s->th ? sec : 4.0 * s->th;
                }
                nxt = nxt > 1.1 * s->th ? nxt : 1.1 * s->th;
                s->pa = s->th;
                s->Da = D;
            } else if (s->hi_nod) {
                nxt = 0.5 * (s->lo + s->hi);   // no slope sign change to interpolate
            } else {
                nxt = s->lo - s->Dlo * (s->hi - s->lo) / (s->Dhi - s->Dlo);
                double w = s->hi - s->lo;
                double a = s->lo + 0.01 * w, b = s->hi - 0.01 * w;
                nxt = nxt < a ? a : (nxt > b ? b : nxt);
            }
            s->th = nxt < 1.5 ? nxt : 1.5;
        }
    }
    if (accept) {
        s->accepted = 1;
        s->ls_active = 0;
        s->theta_prev = s->th;
        for (int k = 0; k < 18; ++k) s->ev_acc[k] = s->ev[k];
        s->mu = s->ev[15] / s->ev[16];
    } else if (failed) {
        s->accepted = 0;
        s->ls_active = 0;
        if (!s->have_prev) {
            s->done = 1;            // no descent along steepest descent either
        } else {
            s->have_prev = 0;       // restart along steepest descent
            s->beta = 0.0;
        }
    } else {
        s->cs[0] = cos(s->th);
        s->cs[1] = sin(s->th);
        s->csf[0] = (float)s->cs[0];
        s->csf[1] = (float)s->cs[1];
    }
    set_cond(ls, use, s->ls_active ? 1u : 0u);
}

}  // namespace

void launch_ctl_norm(CgState *s, cudaStream_t st) { k_ctl_norm<<<1, 1, 0, st>>>(s); }
void launch_ctl_init(CgState *s, cudaStream_t st) { k_ctl_init<<<1, 1, 0, st>>>(s); }
void launch_ctl_grad(CgState *s, int first, cudaGraphConditionalHandle outer, int use_cond, cudaStream_t st)
{
    k_ctl_grad<<<1, 1, 0, st>>>(s, first, outer, use_cond);
}
void launch_ctl_dir(CgState *s, cudaStream_t st) { k_ctl_dir<<<1, 1, 0, st>>>(s); }
void launch_ctl_dhat(CgState *s, cudaGraphConditionalHandle ls, int use_cond, cudaStream_t st)
{
    k_ctl_dhat<<<1, 1, 0, st>>>(s, ls, use_cond);
}
void launch_ctl_ls(CgState *s, cudaGraphConditionalHandle ls, int use_cond, cudaStream_t st)
{
    k_ctl_ls<<<1, 1, 0, st>>>(s, ls, use_cond);
}

}  // namespace ofdft
