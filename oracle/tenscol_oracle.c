/*
 * TensCol reference oracle -- TEST INFRASTRUCTURE ONLY (see tenscol_oracle.h).
 *
 * Plain FP64, single thread, adjacency lists.  Each function restates one
 * step of Algorithm 1 of Goudet, Duval, Hao (TensCol) in the paper's order and
 * notation.  Matrix products against the one-hot tensor S are written as
 * the sums they reduce to (a product with a one-hot column keeps exactly the
 * terms whose row has that colour); nothing is blocked, fused or reordered
 * beyond that.  Readings of points the paper leaves open:
 *   - argmax ties go to the lowest colour index, argmin ties to the lowest d;
 *   - kappa and varpi sum over ordered pairs (every edge twice), as the
 *     double sums of eq. 5 and eq. 6 are written;
 *   - \bar A = J - A keeps its diagonal (bonus_diag = 1) unless disabled;
 *   - c2 = ceil(n / k), so c1 == c2 when k divides n (Section 3.5);
 *   - smoothing (eq. 8) follows the update of iteration t when (t + 1) is a
 *     multiple of nb_iter; 0^x = 0 for the exponents x > 0 used here.
 */
#include "tenscol_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EBADARG (-1)
#define ORC_EGRAPH (-2)
#define ORC_ENOMEM (-3)

int orc_validate_graph(int n, const int *adj_off, const int *adj)
{
    if (n < 0 || (n > 0 && (!adj_off)))
        return ORC_EBADARG;
    if (n == 0)
        return 0;
    if (adj_off[0] != 0)
        return ORC_EGRAPH;
    for (int i = 0; i < n; ++i) {
        if (adj_off[i + 1] < adj_off[i])
            return ORC_EGRAPH;
        for (int e = adj_off[i]; e < adj_off[i + 1]; ++e) {
            int m = adj[e];
            if (m < 0 || m >= n || m == i)
                return ORC_EGRAPH;
            for (int f = adj_off[i]; f < e; ++f)
                if (adj[f] == m)
                    return ORC_EGRAPH; /* duplicate */
            int back = 0; /* the edge must be listed from m's side too */
            for (int f = adj_off[m]; f < adj_off[m + 1]; ++f)
                if (adj[f] == i) {
                    back = 1;
                    break;
                }
            if (!back)
                return ORC_EGRAPH;
        }
    }
    return 0;
}

/* Step 1 (Section 3.4): s_{d,i,j} = 1 iff j = argmax_l w_{d,i,l}. */
int orc_assign(int D, int n, int k, const double *W, int *colors)
{
    if (D < 0 || n < 0 || k < 1 || !W || !colors)
        return ORC_EBADARG;
    for (int d = 0; d < D; ++d)
        for (int i = 0; i < n; ++i) {
            const double *w = W + ((size_t)d * n + i) * k;
            int best = 0;
            for (int j = 1; j < k; ++j)
                if (w[j] > w[best])
                    best = j; /* strict: the first maximum wins */
            colors[(size_t)d * n + i] = best;
        }
    return 0;
}

/* A . S_d: the gamma matrix of the footnote to eq. 13. */
int orc_gamma(int D, int n, int k, const int *adj_off, const int *adj,
              const int *colors, int *Gamma)
{
    if (D < 0 || n < 0 || k < 1 || !colors || !Gamma)
        return ORC_EBADARG;
    memset(Gamma, 0, sizeof(int) * (size_t)D * n * k);
    for (int d = 0; d < D; ++d)
        for (int i = 0; i < n; ++i) {
            int *row = Gamma + ((size_t)d * n + i) * k;
            for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
                row[colors[(size_t)d * n + adj[e]]] += 1;
        }
    return 0;
}

/* Step 2 (eq. 1-2): c_{d,i,m} = a_{i,m} m_{d,i,m}; f_color = half the sum. */
int orc_fitness(int D, int n, int k, const int *adj_off, const int *adj,
                const int *colors, int *gamma_own, long long *f_color)
{
    if (D < 0 || n < 0 || k < 1 || !colors)
        return ORC_EBADARG;
    for (int d = 0; d < D; ++d) {
        long long twice = 0;
        const int *c = colors + (size_t)d * n;
        for (int i = 0; i < n; ++i) {
            int g = 0;
            for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
                g += (c[adj[e]] == c[i]);
            if (gamma_own)
                gamma_own[(size_t)d * n + i] = g;
            twice += g;
        }
        if (f_color)
            f_color[d] = twice / 2;
    }
    return 0;
}

/* k-partitioning fitness (Section 6): M_d replaced by \bar M_d = J - M_d,
 * f(S_d) = 1/2 sum(A (.) \bar M_d) = edges whose ends lie in different
 * groups (cut edges), counted here directly from the adjacency lists. */
int orc_cut(int D, int n, const int *adj_off, const int *adj, const int *colors, long long *cut)
{
    if (D < 0 || n < 0 || !colors || !cut)
        return ORC_EBADARG;
    for (int d = 0; d < D; ++d) {
        long long twice = 0;
        const int *c = colors + (size_t)d * n;
        for (int i = 0; i < n; ++i)
            for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
                twice += (c[adj[e]] != c[i]);
        cut[d] = twice / 2;
    }
    return 0;
}

/* Minimum sum colouring (Section 6): the additive fitness sums the cost of
 * the colour each vertex takes, f_mscp(S_d) = sum_i sum_l s_{d,i,l} z_l. */
int orc_mscp(int D, int n, int k, const int *colors, const int *z, long long *f_mscp)
{
    if (D < 0 || n < 0 || k < 1 || !colors || !f_mscp)
        return ORC_EBADARG;
    for (int d = 0; d < D; ++d) {
        long long f = 0;
        for (int i = 0; i < n; ++i) {
            const int l = colors[(size_t)d * n + i];
            f += z ? (long long)z[l] : (long long)(l + 1);
        }
        f_mscp[d] = f;
    }
    return 0;
}

/* Equity fitness (eq. 3) and its gradient (eq. 14). */
int orc_equity(int D, int n, int k, const int *colors,
               int *sizes, long long *f_eq, int *E)
{
    if (D < 0 || n < 0 || k < 1 || !colors)
        return ORC_EBADARG;
    const int c1 = n / k;
    const int c2 = (n + k - 1) / k;
    int *cnt = (int *)malloc(sizeof(int) * (size_t)k);
    if (!cnt)
        return ORC_ENOMEM;
    for (int d = 0; d < D; ++d) {
        memset(cnt, 0, sizeof(int) * (size_t)k);
        for (int i = 0; i < n; ++i)
            cnt[colors[(size_t)d * n + i]] += 1;
        long long f = 0;
        for (int j = 0; j < k; ++j) {
            int a = abs(cnt[j] - c1), b = abs(cnt[j] - c2);
            f += (a < b) ? a : b;
            if (sizes)
                sizes[(size_t)d * k + j] = cnt[j];
            if (E)
                E[(size_t)d * k + j] = cnt[j] > c2 ? 1 : (cnt[j] < c1 ? -1 : 0);
        }
        if (f_eq)
            f_eq[d] = f;
    }
    free(cnt);
    return 0;
}

/* Step 3-i (eq. 4): \tilde M = sum_d S_d S_d^T. */
int orc_mtilde(int D, int n, const int *colors, int *Mt)
{
    if (D < 0 || n < 0 || !colors || !Mt)
        return ORC_EBADARG;
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) {
            int s = 0;
            for (int d = 0; d < D; ++d)
                s += (colors[(size_t)d * n + i] == colors[(size_t)d * n + m]);
            Mt[(size_t)i * n + m] = s;
        }
    return 0;
}

/* The k-partitioning counterpart of eq. 4 (Section 6: M replaced by
 * \bar M = J - M): Mb[i*n+m] = sum_d (1 - m_{d,i,m}) = #{d : c_d(i) != c_d(m)};
 * Mb[i*n+i] = 0. */
int orc_mbar(int D, int n, const int *colors, int *Mb)
{
    if (D < 0 || n < 0 || !colors || !Mb)
        return ORC_EBADARG;
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) {
            int s = 0;
            for (int d = 0; d < D; ++d)
                s += (colors[(size_t)d * n + i] != colors[(size_t)d * n + m]);
            Mb[(size_t)i * n + m] = s;
        }
    return 0;
}

/* Marks the neighbours of i in mark[] (1) and returns nothing. */
static void mark_row(int i, const int *adj_off, const int *adj, unsigned char *mark, int v)
{
    for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
        mark[adj[e]] = (unsigned char)v;
}

/* eq. 5 (kappa) and eq. 6 (varpi), ordered pairs. */
int orc_penalty_bonus(int n, const int *adj_off, const int *adj, const int *Mt,
                      double alpha, double beta, int bonus_diag,
                      double *kappa, double *varpi)
{
    if (n < 0 || !Mt)
        return ORC_EBADARG;
    unsigned char *mark = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!mark)
        return ORC_ENOMEM;
    /* Mt holds integers in [0, D]; tabulate x^alpha, x^beta once */
    int vmax = 0;
    for (size_t q = 0; q < (size_t)n * n; ++q)
        if (Mt[q] > vmax)
            vmax = Mt[q];
    double *pa = (double *)malloc(sizeof(double) * (size_t)(vmax + 1));
    double *pb = (double *)malloc(sizeof(double) * (size_t)(vmax + 1));
    if (!pa || !pb) {
        free(mark); free(pa); free(pb);
        return ORC_ENOMEM;
    }
    for (int x = 0; x <= vmax; ++x) {
        pa[x] = pow((double)x, alpha);
        pb[x] = pow((double)x, beta);
    }
    double ks = 0.0, vs = 0.0;
    for (int i = 0; i < n; ++i) {
        mark_row(i, adj_off, adj, mark, 1);
        for (int m = 0; m < n; ++m) {
            int mt = Mt[(size_t)i * n + m];
            if (mark[m])
                ks += pa[mt];
            else if (m != i || bonus_diag)
                vs += pb[mt];
        }
        mark_row(i, adj_off, adj, mark, 0);
    }
    free(mark); free(pa); free(pb);
    if (kappa)
        *kappa = ks;
    if (varpi)
        *varpi = vs;
    return 0;
}

/* eq. 13: grad_S L = A.S + nu t grad f_eq + 2 alpha lambda t (A (.) Mt^(alpha-1)).S
 *                    - 2 beta mu t (\bar A (.) Mt^(beta-1)).S
 * k-partitioning (problem 2 or 3, Section 6): every M_d of eq. 7 becomes
 * J - M_d, so Mt here is \bar M~ = sum_d (J - M_d) (orc_mbar) and, since
 * d(J - M_d)/dS_d = -dM_d/dS_d, every term but the equity one changes sign:
 * grad_S L = -A.S + nu t grad f_eq - 2 alpha lambda t (A (.) Mt^(alpha-1)).S
 *            + 2 beta mu t (\bar A (.) Mt^(beta-1)).S                           */
int orc_grad_S(int D, int n, int k, const int *adj_off, const int *adj,
               const int *colors, const int *Mt, const int *E,
               const orc_params *p, long long t, double *G)
{
    if (D < 0 || n < 0 || k < 1 || !colors || !Mt || !p || !G)
        return ORC_EBADARG;
    const double sg = (p->problem == 2 || p->problem == 3) ? -1.0 : 1.0;
    const double tt = (double)t;
    const double cpen = 2.0 * p->alpha * p->lambda_ * tt;
    const double cbon = 2.0 * p->beta * p->mu * tt;
    const double ceq = p->nu * tt;
    unsigned char *mark = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    /* Mt holds small non-negative integers: tabulate the pair coefficients */
    int vmax = D;
    for (size_t q = 0; q < (size_t)n * n; ++q) {
        if (Mt[q] < 0) {
            free(mark);
            return ORC_EBADARG;
        }
        if (Mt[q] > vmax)
            vmax = Mt[q];
    }
    double *ca = (double *)malloc(sizeof(double) * (size_t)(vmax + 1));
    double *cb = (double *)malloc(sizeof(double) * (size_t)(vmax + 1));
    if (!mark || !ca || !cb) {
        free(mark); free(ca); free(cb);
        return ORC_ENOMEM;
    }
    for (int x = 0; x <= vmax; ++x) {
        ca[x] = cpen * pow((double)x, p->alpha - 1.0);
        cb[x] = cbon * pow((double)x, p->beta - 1.0);
    }
    for (int i = 0; i < n; ++i) {
        mark_row(i, adj_off, adj, mark, 1);
        for (int d = 0; d < D; ++d) {
            const int *c = colors + (size_t)d * n;
            double *g = G + ((size_t)d * n + i) * k;
            for (int j = 0; j < k; ++j)
                g[j] = 0.0;
            /* (A . S_d)[i, j]: one count per neighbour of colour j */
            for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
                g[c[adj[e]]] += sg;
            /* nu t d f_eq / d s_{d,i,j} (eq. 14), the same for every vertex */
            if (E && ceq != 0.0)
                for (int j = 0; j < k; ++j)
                    g[j] += ceq * (double)E[(size_t)d * k + j];
            /* penalisation and bonus products with S_d: every vertex m adds
             * its pair coefficient to the column of its own colour */
            for (int m = 0; m < n; ++m) {
                int mt = Mt[(size_t)i * n + m];
                if (mark[m]) {
                    if (cpen != 0.0)
                        g[c[m]] += sg * ca[mt];
                } else if (m != i || p->bonus_diag) {
                    if (cbon != 0.0)
                        g[c[m]] -= sg * cb[mt];
                }
            }
        }
        mark_row(i, adj_off, adj, mark, 0);
    }
    free(mark); free(ca); free(cb);
    return 0;
}

/* Step 4: softmax (eq. 10-11), straight-through gradient (eq. 12),
 * descent step, and the periodic smoothing of eq. 8. */
int orc_update(int D, int n, int k, const orc_params *p, long long t,
               const double *G, double *W, double *gW)
{
    if (D < 0 || n < 0 || k < 1 || !p || !G || !W || p->nb_iter < 1)
        return ORC_EBADARG;
    const int smooth = ((t + 1) % p->nb_iter) == 0;
    double *s = (double *)malloc(sizeof(double) * (size_t)k);
    if (!s)
        return ORC_ENOMEM;
    for (size_t r = 0; r < (size_t)D * n; ++r) {
        double *w = W + r * k;
        const double *g = G + r * k;
        double mx = w[0];
        for (int j = 1; j < k; ++j)
            if (w[j] > mx)
                mx = w[j];
        double z = 0.0;
        for (int j = 0; j < k; ++j) {
            s[j] = exp(w[j] - mx);
            z += s[j];
        }
        double dot = 0.0; /* (S^ (.) grad_S L) . J, one value per row */
        for (int j = 0; j < k; ++j) {
            s[j] /= z;
            dot += s[j] * g[j];
        }
        for (int j = 0; j < k; ++j) {
            double gw = s[j] * (g[j] - dot);
            if (gW)
                gW[r * k + j] = gw;
            w[j] -= p->eta * gw;
            if (smooth)
                w[j] /= p->rho;
        }
    }
    free(s);
    return 0;
}

int orc_step(int D, int n, int k, const int *adj_off, const int *adj,
             const orc_params *p, long long t, int stop_on_legal,
             double *W,
             int *colors, int *gamma_own, long long *f_color, long long *f_eq,
             long long *f_cut, long long *f_mscp, int *Mt, double *G, double *gW,
             double *loss, double *kappa, double *varpi,
             long long *f_min, int *d_star, int *updated)
{
    if (D < 1 || n < 0 || k < 1 || !p || !W || p->problem < 0 || p->problem > 4)
        return ORC_EBADARG;
    if (p->zcost)
        for (int l = 0; l < k; ++l)
            if (p->zcost[l] < 0)
                return ORC_EBADARG;
    const int mscp = p->problem == 4; /* minimum sum colouring */
    const int part = p->problem == 2 || p->problem == 3; /* k-partitioning */
    const size_t Dn = (size_t)D * n, Dk = (size_t)D * k, nn = (size_t)n * n;
    int rc = 0;
    int *c = colors ? colors : (int *)malloc(sizeof(int) * (Dn ? Dn : 1));
    long long *fc = f_color ? f_color : (long long *)malloc(sizeof(long long) * D);
    long long *fe = f_eq ? f_eq : (long long *)malloc(sizeof(long long) * D);
    long long *fx = f_cut ? f_cut : (long long *)malloc(sizeof(long long) * D);
    long long *fm = f_mscp ? f_mscp : (long long *)malloc(sizeof(long long) * D);
    int *E = (int *)malloc(sizeof(int) * (Dk ? Dk : 1));
    int *M = Mt ? Mt : (int *)malloc(sizeof(int) * (nn ? nn : 1));
    int *Mb = part ? (int *)malloc(sizeof(int) * (nn ? nn : 1)) : NULL;
    double *Gr = G ? G : (double *)malloc(sizeof(double) * (Dn * k > 0 ? Dn * k : 1));
    if (!c || !fc || !fe || !fx || !fm || !E || !M || (part && !Mb) || !Gr) {
        rc = ORC_ENOMEM;
        goto out;
    }
    /* Step 1 */
    orc_assign(D, n, k, W, c);
    /* Step 2 */
    orc_fitness(D, n, k, adj_off, adj, c, gamma_own, fc);
    orc_cut(D, n, adj_off, adj, c, fx);
    orc_equity(D, n, k, c, NULL, fe, E);
    orc_mscp(D, n, k, c, p->zcost, fm);
    if (mscp) /* f_mscp replaces f_eq: its gradient z_l stands in for eq. 14 */
        for (int d = 0; d < D; ++d)
            for (int j = 0; j < k; ++j)
                E[(size_t)d * k + j] = p->zcost ? p->zcost[j] : j + 1;
    /* the fitness each problem minimises: f_color (k-COL), f_color + f_eq
     * (ECP), cut edges (k-partitioning), cut edges + f_eq (balanced),
     * f_color + f_mscp (minimum sum colouring) */
    long long *fobj = part ? fx : fc;
    long long *fadd = mscp ? fm : fe; /* the additive term of the fitness and of eq. 7 */
    const int with_add = p->problem == 1 || p->problem == 3 || mscp;
    long long fmin = -1;
    int dstar = 0;
    for (int d = 0; d < D; ++d) {
        long long f = fobj[d] + (with_add ? fadd[d] : 0);
        if (fmin < 0 || f < fmin) {
            fmin = f;
            dstar = d;
        }
    }
    if (f_min)
        *f_min = fmin;
    if (d_star)
        *d_star = dstar;
    /* Step 3 (the partitioning terms use \bar M~ in place of M~) */
    orc_mtilde(D, n, c, M);
    if (part)
        orc_mbar(D, n, c, Mb);
    const int *X = part ? Mb : M;
    double ks = 0.0, vs = 0.0;
    orc_penalty_bonus(n, adj_off, adj, X, p->alpha, p->beta, p->bonus_diag, &ks, &vs);
    {
        double sc = 0.0, se = 0.0;
        for (int d = 0; d < D; ++d) {
            sc += (double)fobj[d];
            se += (double)fadd[d];
        }
        const double tt = (double)t;
        if (loss)
            *loss = sc + p->nu * tt * se + p->lambda_ * tt * ks - p->mu * tt * vs;
        if (kappa)
            *kappa = ks;
        if (varpi)
            *varpi = vs;
    }
    orc_grad_S(D, n, k, adj_off, adj, c, X, E, p, t, Gr);
    /* Step 4 unless the population already holds a legal solution */
    if (stop_on_legal && fmin == 0) {
        if (updated)
            *updated = 0;
        if (gW)
            memset(gW, 0, sizeof(double) * Dn * k);
    } else {
        rc = orc_update(D, n, k, p, t, Gr, W, gW);
        if (updated)
            *updated = 1;
    }
out:
    if (c != colors) free(c);
    if (fc != f_color) free(fc);
    if (fe != f_eq) free(fe);
    if (fx != f_cut) free(fx);
    if (fm != f_mscp) free(fm);
    free(Mb);
    free(E);
    if (M != Mt) free(M);
    if (Gr != G) free(Gr);
    return rc;
}

long long orc_run(int D, int n, int k, const int *adj_off, const int *adj,
                  const orc_params *p, long long *t, long long max_iter,
                  int stop_on_legal, double *W,
                  int *best_colors, long long *best_f, long long *best_t)
{
    if (D < 1 || n < 0 || k < 1 || !p || !t || !W || max_iter < 0)
        return ORC_EBADARG;
    int *c = (int *)malloc(sizeof(int) * ((size_t)D * n > 0 ? (size_t)D * n : 1));
    if (!c)
        return ORC_ENOMEM;
    long long done = 0;
    long long bf = best_f ? *best_f : -1;
    for (long long it = 0; it < max_iter; ++it) {
        long long fmin = 0;
        int dstar = 0, upd = 0;
        int rc = orc_step(D, n, k, adj_off, adj, p, *t, stop_on_legal, W, c,
                          NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL,
                          &fmin, &dstar, &upd);
        if (rc) {
            free(c);
            return rc;
        }
        if (bf < 0 || fmin < bf) {
            bf = fmin;
            if (best_colors)
                memcpy(best_colors, c + (size_t)dstar * n, sizeof(int) * (size_t)n);
            if (best_t)
                *best_t = *t;
        }
        if (!upd)
            break;
        *t += 1;
        ++done;
    }
    if (best_f)
        *best_f = bf;
    free(c);
    return done;
}

int orc_relaxed(int D, int n, int k, const int *adj_off, const int *adj,
                const orc_params *p, long long t, double tau, const double *W,
                double *loss, double *gradW, double *Mt)
{
    if (D < 1 || n < 1 || k < 1 || !p || !W || !(tau > 0.0))
        return ORC_EBADARG;
    const size_t Dnk = (size_t)D * n * k, nn = (size_t)n * n;
    double *S = (double *)malloc(sizeof(double) * Dnk);
    double *M = (double *)calloc(nn, sizeof(double));
    double *Bp = (double *)malloc(sizeof(double) * nn);
    unsigned char *mark = (unsigned char *)calloc((size_t)n, 1);
    if (!S || !M || !Bp || !mark) {
        free(S); free(M); free(Bp); free(mark);
        return ORC_ENOMEM;
    }
    /* S = softmax(W / tau) over colours */
    for (size_t r = 0; r < (size_t)D * n; ++r) {
        const double *w = W + r * k;
        double mx = w[0] / tau;
        for (int j = 1; j < k; ++j)
            if (w[j] / tau > mx)
                mx = w[j] / tau;
        double z = 0.0;
        for (int j = 0; j < k; ++j) {
            S[r * k + j] = exp(w[j] / tau - mx);
            z += S[r * k + j];
        }
        for (int j = 0; j < k; ++j)
            S[r * k + j] /= z;
    }
    /* eq. 4 with M_d = S_d S_d^T */
    for (int d = 0; d < D; ++d)
        for (int i = 0; i < n; ++i)
            for (int m = 0; m < n; ++m) {
                const double *a = S + ((size_t)d * n + i) * k, *b = S + ((size_t)d * n + m) * k;
                double dot = 0.0;
                for (int j = 0; j < k; ++j)
                    dot += a[j] * b[j];
                M[(size_t)i * n + m] += dot;
            }
    /* loss (eq. 7) and the pair coefficients of eq. 13 */
    const double tt = (double)t;
    double fc = 0.0, ks = 0.0, vs = 0.0;
    for (int i = 0; i < n; ++i) {
        mark_row(i, adj_off, adj, mark, 1);
        for (int m = 0; m < n; ++m) {
            const double x = M[(size_t)i * n + m];
            double b = 0.0;
            if (mark[m]) {
                fc += 0.5 * x;
                ks += pow(x, p->alpha);
                b = 1.0 + 2.0 * p->alpha * p->lambda_ * tt * pow(x, p->alpha - 1.0);
            } else if (m != i || p->bonus_diag) {
                vs += pow(x, p->beta);
                b = -2.0 * p->beta * p->mu * tt * pow(x, p->beta - 1.0);
            }
            Bp[(size_t)i * n + m] = b;
        }
        mark_row(i, adj_off, adj, mark, 0);
    }
    if (loss)
        *loss = fc + p->lambda_ * tt * ks - p->mu * tt * vs;
    if (gradW) {
        /* grad_S L = B' . S_d (eq. 13), then the softmax Jacobian / tau */
        double *g = (double *)malloc(sizeof(double) * (size_t)k);
        if (!g) {
            free(S); free(M); free(Bp); free(mark);
            return ORC_ENOMEM;
        }
        for (int d = 0; d < D; ++d)
            for (int i = 0; i < n; ++i) {
                for (int j = 0; j < k; ++j)
                    g[j] = 0.0;
                for (int m = 0; m < n; ++m) {
                    const double b = Bp[(size_t)i * n + m];
                    const double *sm = S + ((size_t)d * n + m) * k;
                    for (int j = 0; j < k; ++j)
                        g[j] += b * sm[j];
                }
                const double *si = S + ((size_t)d * n + i) * k;
                double dot = 0.0;
                for (int j = 0; j < k; ++j)
                    dot += si[j] * g[j];
                double *gw = gradW + ((size_t)d * n + i) * k;
                for (int j = 0; j < k; ++j)
                    gw[j] = si[j] * (g[j] - dot) / tau;
            }
        free(g);
    }
    if (Mt)
        memcpy(Mt, M, sizeof(double) * nn);
    free(S); free(M); free(Bp); free(mark);
    return 0;
}

/* Multicolouring, Step 1 (Section 6): the demand[i] largest weights of w_{d,i},
 * picked one at a time as the largest not yet taken (lowest index on ties). */
int orc_assign_multi(int D, int n, int k, const double *W, const int *demand, double *S)
{
    if (D < 0 || n < 0 || k < 1 || !W || !demand || !S)
        return ORC_EBADARG;
    for (int i = 0; i < n; ++i)
        if (demand[i] < 1 || demand[i] > k)
            return ORC_EBADARG;
    memset(S, 0, sizeof(double) * (size_t)D * n * k);
    for (size_t r = 0; r < (size_t)D * n; ++r) {
        const double *w = W + r * k;
        double *s = S + r * k;
        const int c = demand[r % (size_t)n];
        for (int q = 0; q < c; ++q) {
            int best = -1;
            for (int l = 0; l < k; ++l)
                if (s[l] == 0.0 && (best < 0 || w[l] > w[best]))
                    best = l;
            s[best] = 1.0;
        }
    }
    return 0;
}

int orc_step_multi(int D, int n, int k, const int *adj_off, const int *adj, const int *demand,
                   const orc_params *p, long long t, int stop_on_legal, double *W,
                   double *S, long long *f_color, int *Mt, double *G, double *gW,
                   double *loss, double *kappa, double *varpi,
                   long long *f_min, int *d_star, int *updated)
{
    if (D < 1 || n < 0 || k < 1 || !p || !W || !demand || p->problem != 0)
        return ORC_EBADARG;
    const size_t Dn = (size_t)D * n, nn = (size_t)n * n;
    int rc = 0;
    double *Sx = S ? S : (double *)malloc(sizeof(double) * (Dn * k > 0 ? Dn * k : 1));
    double *A = (double *)calloc(nn ? nn : 1, sizeof(double));
    double *Md = (double *)malloc(sizeof(double) * (nn ? nn : 1)); /* M_d of one individual */
    double *Mtd = (double *)calloc(nn ? nn : 1, sizeof(double));  /* M~ */
    long long *fc = f_color ? f_color : (long long *)malloc(sizeof(long long) * D);
    double *Gr = G ? G : (double *)malloc(sizeof(double) * (Dn * k > 0 ? Dn * k : 1));
    if (!Sx || !A || !Md || !Mtd || !fc || !Gr) {
        rc = ORC_ENOMEM;
        goto out;
    }
    if ((rc = orc_assign_multi(D, n, k, W, demand, Sx)))
        goto out;
    for (int i = 0; i < n; ++i)
        for (int e = adj_off[i]; e < adj_off[i + 1]; ++e)
            A[(size_t)i * n + adj[e]] = 1.0;
    /* Step 2: M_d = S_d S_d^T, f_color = 1/2 sum(A (.) M_d); Step 3-i: M~ */
    for (int d = 0; d < D; ++d) {
        const double *Sd = Sx + (size_t)d * n * k;
        double twice = 0.0;
        for (int i = 0; i < n; ++i)
            for (int m = 0; m < n; ++m) {
                double v = 0.0;
                for (int l = 0; l < k; ++l)
                    v += Sd[(size_t)i * k + l] * Sd[(size_t)m * k + l];
                Md[(size_t)i * n + m] = v;
                twice += A[(size_t)i * n + m] * v;
                Mtd[(size_t)i * n + m] += v;
            }
        fc[d] = (long long)(twice / 2.0 + 0.5);
    }
    long long fmin = -1;
    int dstar = 0;
    for (int d = 0; d < D; ++d)
        if (fmin < 0 || fc[d] < fmin) {
            fmin = fc[d];
            dstar = d;
        }
    if (f_min)
        *f_min = fmin;
    if (d_star)
        *d_star = dstar;
    if (Mt)
        for (size_t q = 0; q < nn; ++q)
            Mt[q] = (int)(Mtd[q] + 0.5);
    /* eq. 5-7 */
    const double tt = (double)t;
    double ks = 0.0, vs = 0.0, sc = 0.0;
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) {
            const double a = A[(size_t)i * n + m], x = Mtd[(size_t)i * n + m];
            const double abar = (m == i && !p->bonus_diag) ? 0.0 : 1.0 - a;
            ks += a * pow(x, p->alpha);
            vs += abar * pow(x, p->beta);
        }
    for (int d = 0; d < D; ++d)
        sc += (double)fc[d];
    if (loss)
        *loss = sc + p->lambda_ * tt * ks - p->mu * tt * vs;
    if (kappa)
        *kappa = ks;
    if (varpi)
        *varpi = vs;
    /* eq. 13, row by row: G_d[i,j] = sum_m C_im S_d[m,j] with the pair
     * coefficient C_im = a_im (1 + 2 alpha lambda t m~^(alpha-1))
     *                   - abar_im 2 beta mu t m~^(beta-1) */
    for (int d = 0; d < D; ++d) {
        const double *Sd = Sx + (size_t)d * n * k;
        for (int i = 0; i < n; ++i) {
            double *g = Gr + ((size_t)d * n + i) * k;
            for (int j = 0; j < k; ++j)
                g[j] = 0.0;
            for (int m = 0; m < n; ++m) {
                const double a = A[(size_t)i * n + m], x = Mtd[(size_t)i * n + m];
                const double abar = (m == i && !p->bonus_diag) ? 0.0 : 1.0 - a;
                double cim = a;
                if (a != 0.0)
                    cim += 2.0 * p->alpha * p->lambda_ * tt * pow(x, p->alpha - 1.0);
                if (abar != 0.0)
                    cim -= 2.0 * p->beta * p->mu * tt * pow(x, p->beta - 1.0);
                if (cim == 0.0)
                    continue;
                for (int j = 0; j < k; ++j)
                    g[j] += cim * Sd[(size_t)m * k + j];
            }
        }
    }
    /* Step 4 unless the population already holds a legal multicolouring */
    if (stop_on_legal && fmin == 0) {
        if (updated)
            *updated = 0;
        if (gW)
            memset(gW, 0, sizeof(double) * Dn * k);
    } else {
        rc = orc_update(D, n, k, p, t, Gr, W, gW);
        if (updated)
            *updated = 1;
    }
out:
    if (Sx != S) free(Sx);
    if (fc != f_color) free(fc);
    if (Gr != G) free(Gr);
    free(A);
    free(Md);
    free(Mtd);
    return rc;
}

long long orc_check_conflicts(long long n_edges, const int *u, const int *v,
                              const int *coloring)
{
    if (n_edges < 0 || (n_edges > 0 && (!u || !v || !coloring)))
        return ORC_EBADARG;
    long long bad = 0;
    for (long long e = 0; e < n_edges; ++e)
        bad += (coloring[u[e]] == coloring[v[e]]);
    return bad;
}

long long orc_check_equity(int n, int k, const int *coloring)
{
    if (n < 0 || k < 1 || (n > 0 && !coloring))
        return ORC_EBADARG;
    long long f = 0;
    int *cnt = (int *)calloc((size_t)k, sizeof(int));
    if (!cnt)
        return ORC_ENOMEM;
    for (int i = 0; i < n; ++i) {
        if (coloring[i] < 0 || coloring[i] >= k) {
            free(cnt);
            return ORC_EBADARG;
        }
        cnt[coloring[i]] += 1;
    }
    const int c1 = n / k, c2 = (n + k - 1) / k;
    for (int j = 0; j < k; ++j) {
        int a = abs(cnt[j] - c1), b = abs(cnt[j] - c2);
        f += (a < b) ? a : b;
    }
    free(cnt);
    return f;
}
