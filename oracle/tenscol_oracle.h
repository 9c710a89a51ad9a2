/*
 * TensCol reference oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of one iteration of the
 * population-based gradient-descent weight learning for graph coloring
 * (Goudet, Duval, Hao, "Population-based gradient descent weight learning
 * for graph coloring problems", Section 3 and Algorithm 1), over adjacency
 * lists.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (all buffers are caller-owned host memory):
 *   graph   : n vertices, adjacency lists adj_off[n+1] / adj[adj_off[n]]
 *             (symmetric, no self loops, neighbour ids in [0, n)).
 *   W       : D*n*k doubles, index (d*n + i)*k + j  (w_{d,i,j}, Section 3.2)
 *   colors  : D*n ints, c_d(i) in [0, k)
 *   Mt      : n*n ints, \tilde m_{i,m} (eq. 4)
 * Every function returns 0 on success and a negative value on bad input.
 */
#ifndef TENSCOL_ORACLE_H
#define TENSCOL_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int problem;        /* 0 = k-COL (GCP), 1 = ECP, 2 = k-partitioning,
                           3 = balanced k-partitioning, 4 = minimum sum
                           colouring (Section 6)                            */
    double sigma0;      /* std of the N(0, sigma0) initial weights (Table 2) */
    double eta;         /* learning rate                                      */
    double alpha;       /* penalisation exponent  (eq. 5)                     */
    double lambda_;     /* penalisation weight    (eq. 7)                     */
    double beta;        /* bonus exponent         (eq. 6)                     */
    double mu;          /* bonus weight           (eq. 7)                     */
    double nu;          /* equity weight          (eq. 7)                     */
    double rho;         /* smoothing divisor      (eq. 8)                     */
    int nb_iter;        /* smoothing period       (Step 4-iv)                 */
    int bonus_diag;     /* 1: \bar A = J - A keeps its diagonal (Section 3.6.2)*/
    const int *zcost;   /* problem 4: cost z_l >= 0 of colour l (k entries);
                           NULL: z_l = l + 1 (colours numbered 1..k)        */
} orc_params;

/* Structural check of the adjacency lists: ids in range, no self loop,
 * every edge listed in both directions, no duplicates. 0 if valid. */
int orc_validate_graph(int n, const int *adj_off, const int *adj);

/* Step 1: c_d(i) = lowest j with w_{d,i,j} maximal (Section 3.4). */
int orc_assign(int D, int n, int k, const double *W, int *colors);

/* Gamma = A . S_d  (footnote to eq. 13): Gamma[(d*n+i)*k+j] = number of
 * neighbours of i with colour j in individual d. */
int orc_gamma(int D, int n, int k, const int *adj_off, const int *adj,
              const int *colors, int *Gamma);

/* Step 2 (eq. 1): gamma_own[d*n+i] = conflicting neighbours of i,
 * f_color[d] = half their sum = monochromatic edges of individual d. */
int orc_fitness(int D, int n, int k, const int *adj_off, const int *adj,
                const int *colors, int *gamma_own, long long *f_color);

/* k-partitioning fitness (Section 6): cut[d] = edges whose ends lie in
 * different groups of individual d, 1/2 sum(A (.) (J - M_d)). */
int orc_cut(int D, int n, const int *adj_off, const int *adj, const int *colors, long long *cut);

/* Equity (eq. 3, eq. 14): sizes[d*k+j] = #V_{d,j}; f_eq[d]; E[d*k+j] in
 * {-1,0,+1} = d f_eq / d s_{d,i,j}.  c1 = floor(n/k), c2 = ceil(n/k). */
int orc_equity(int D, int n, int k, const int *colors,
               int *sizes, long long *f_eq, int *E);

/* Step 3-i (eq. 4): Mt[i*n+m] = #{d : c_d(i) == c_d(m)}; Mt[i*n+i] = D. */
int orc_mtilde(int D, int n, const int *colors, int *Mt);

/* Minimum sum colouring (Section 6): f_mscp[d] = sum_i sum_l s_{d,i,l} z_l =
 * the total cost of the colours individual d uses (z = NULL: z_l = l + 1). */
int orc_mscp(int D, int n, int k, const int *colors, const int *z, long long *f_mscp);

/* k-partitioning counterpart of eq. 4 (Section 6, M -> J - M):
 * Mb[i*n+m] = #{d : c_d(i) != c_d(m)}; Mb[i*n+i] = 0. */
int orc_mbar(int D, int n, const int *colors, int *Mb);

/* eq. 5 and eq. 6 over ordered pairs (i, m):
 * kappa = sum a_im Mt^alpha, varpi = sum (1 - a_im) Mt^beta
 * (diagonal of \bar A included iff bonus_diag). */
int orc_penalty_bonus(int n, const int *adj_off, const int *adj, const int *Mt,
                      double alpha, double beta, int bonus_diag,
                      double *kappa, double *varpi);

/* eq. 13: grad_S L for the one-hot population at iteration t, D*n*k.  For
 * the k-partitioning problems (2, 3) Mt must be \bar M~ (orc_mbar) and the
 * A.S, penalty and bonus terms change sign (derivative of eq. 7 with every
 * M_d replaced by J - M_d); the equity term keeps its sign. */
int orc_grad_S(int D, int n, int k, const int *adj_off, const int *adj,
               const int *colors, const int *Mt, const int *E,
               const orc_params *p, long long t, double *G);

/* Step 4 (eq. 10-12, eq. 8): softmax straight-through gradient
 * gW = S^ (.) (G - (S^ (.) G) J), W <- W - eta gW, then W <- W / rho when
 * (t + 1) is a multiple of nb_iter.  gW may be NULL. */
int orc_update(int D, int n, int k, const orc_params *p, long long t,
               const double *G, double *W, double *gW);

/* One full iteration at counter t on W (in/out).  Every output may be NULL.
 * loss = f(S) + nu t f_eq(S) + lambda t kappa - mu t varpi  (eq. 7), with
 * f = f_color (problems 0, 1, 4) or the cut edges f_cut (problems 2, 3,
 * whose kappa and varpi are taken over \bar M~); for problem 4 the additive
 * fitness f_mscp takes the place of f_eq in the loss and the gradient (the
 * derivative of nu t f_mscp by s_{d,i,l} is nu t z_l).  The fitness
 * minimised per individual is f_color (k-COL), f_color + f_eq (ECP), f_cut
 * (k-partitioning), f_cut + f_eq (balanced) or f_color + f_mscp (minimum
 * sum colouring); *f_min, *d_star = lowest d attaining it.  Mt always receives M~ (eq. 4).  If stop_on_legal and
 * f_min == 0 the weights are left untouched and *updated = 0 (Algorithm 1
 * stop rule), else *updated = 1. */
int orc_step(int D, int n, int k, const int *adj_off, const int *adj,
             const orc_params *p, long long t, int stop_on_legal,
             double *W,
             int *colors, int *gamma_own, long long *f_color, long long *f_eq,
             long long *f_cut, long long *f_mscp, int *Mt, double *G, double *gW,
             double *loss, double *kappa, double *varpi,
             long long *f_min, int *d_star, int *updated);

/* Algorithm 1 loop: up to max_iter iterations from counter *t (in/out).
 * Keeps the best-so-far individual (strictly improving f_min, lowest d on
 * ties) in best_colors[n]; stops early on a legal population when
 * stop_on_legal.  Returns iterations performed (updates) or < 0. */
long long orc_run(int D, int n, int k, const int *adj_off, const int *adj,
                  const orc_params *p, long long *t, long long max_iter,
                  int stop_on_legal, double *W,
                  int *best_colors, long long *best_f, long long *best_t);

/* Relaxation used to check gradients (Section 3.8): S = softmax(W / tau)
 * row-wise, real valued, and eq. 7 with its GCP terms evaluated literally on
 * it (M_d = S_d S_d^T, M~ = sum_d M_d, nu = 0):
 *   loss = 1/2 sum_{i,m} a_im M~_im + lambda t kappa - mu t varpi.
 * gradW (may be NULL) = d loss / d W by the chain rule through eq. 13 and
 * the softmax Jacobian with temperature tau.  Also returns M~ if Mt != NULL. */
int orc_relaxed(int D, int n, int k, const int *adj_off, const int *adj,
                const orc_params *p, long long t, double tau, const double *W,
                double *loss, double *gradW, double *Mt);

/* Multicolouring (Section 6): vertex i must take demand[i] >= 1 colours.
 * Step 1 becomes: S_{d,i,l} = 1 for the demand[i] colours l with the largest
 * w_{d,i,l} (the lower index first among equal weights), else 0.  S is the
 * dense D*n*k 0/1 tensor, index (d*n + i)*k + l. */
int orc_assign_multi(int D, int n, int k, const double *W, const int *demand, double *S);

/* One iteration of Algorithm 1 for multicolouring (problem 0 only; the
 * equity term is not used), every quantity from its definition on the dense
 * tensor S of orc_assign_multi: M_d = S_d S_d^T, f_color(S_d) = 1/2
 * sum(A (.) M_d) (eq. 1-2), M~ = sum_d M_d (eq. 4), kappa and varpi (eq. 5-6
 * over ordered pairs, the diagonal of \bar A iff bonus_diag), L (eq. 7),
 * grad_S L = A S_d + 2 alpha lambda t (A (.) M~^(alpha-1)) S_d
 *            - 2 beta mu t (\bar A (.) M~^(beta-1)) S_d  (eq. 13),
 * then Step 4 (orc_update).  Outputs as for orc_step (any may be NULL); S
 * receives the assignment of this iteration. */
int orc_step_multi(int D, int n, int k, const int *adj_off, const int *adj, const int *demand,
                   const orc_params *p, long long t, int stop_on_legal, double *W,
                   double *S, long long *f_color, int *Mt, double *G, double *gW,
                   double *loss, double *kappa, double *varpi,
                   long long *f_min, int *d_star, int *updated);

/* Checker: recount conflicts edge by edge from an edge list (u[e], v[e]),
 * and the equity deviation of a single colouring. */
long long orc_check_conflicts(long long n_edges, const int *u, const int *v,
                              const int *coloring);
long long orc_check_equity(int n, int k, const int *coloring);

#ifdef __cplusplus
}
#endif
#endif
