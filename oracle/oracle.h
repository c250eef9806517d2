/*
 * oracle.h -- C interface of the FP64 CPU oracle (test infrastructure only).
 *
 * The CUDA library never includes this header; see oracle.c for what every
 * function computes and the paper passages it follows.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#define ORA_OK 0
#define ORA_ERR_ARG (-1)
#define ORA_ERR_OOM (-2)

#define ORA_OPEN_BH 0
#define ORA_OPEN_REL 1

typedef struct {
    double box;          /* periodic cube [0, box)^3 */
    double G;
    double eps;          /* Plummer-equivalent softening; h = 2.8 eps */
    double r_s;          /* split scale A_smth; <= 0: no split, no cutoff */
    double rcut_over_rs; /* cutoff radius in units of r_s */
    double theta;        /* Barnes-Hut opening angle */
    double alpha;        /* relative-criterion tolerance */
    double theta_first_pass;
    int32_t opening;
    int32_t leaf_max;
    int32_t group_max;
    int32_t pad;
} ora_params;

typedef struct ora_tree ora_tree;

/* counts */
enum { ORA_N = 0, ORA_NODES, ORA_CHILDREN, ORA_GROUPS, ORA_LIST_LEN };
/* fields */
enum {
    ORA_F_X = 0, ORA_F_Y, ORA_F_Z, ORA_F_KEY, ORA_F_PERM,
    ORA_F_LEVEL, ORA_F_BEG, ORA_F_END, ORA_F_PARENT, ORA_F_CBEG, ORA_F_CCNT, ORA_F_CHILD,
    ORA_F_MASS, ORA_F_COM, ORA_F_MSUM, ORA_F_NEXTNODE, ORA_F_SIBLING, ORA_F_PNEXT,
    ORA_F_GBEG, ORA_F_GEND, ORA_F_GLO, ORA_F_GHI, ORA_F_EXT_S, ORA_F_EXT_L
};

int ora_quantize1(double v, double box, uint32_t *out);
uint64_t ora_morton(uint32_t x, uint32_t y, uint32_t z);
double ora_soft_g(double r, double h);
double ora_split_s(double r, double rs);
double ora_soft_psi(double r, double h);
double ora_split_p(double r, double rs);

int ora_tree_build(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   ora_tree **out);
void ora_tree_free(ora_tree *t);
int ora_tree_refit(ora_tree *t, const double *pos);
int64_t ora_tree_count(const ora_tree *t, int what);
int ora_tree_get(const ora_tree *t, int what, void *dst);
int ora_tree_force(ora_tree *t, const float *a_old, int opening, double theta, double alpha,
                   const int64_t *sel, int64_t nsel, double *acc, uint32_t *npp,
                   uint32_t *npn, int keep_lists, int nthreads);
int ora_tree_force_pot(ora_tree *t, const float *a_old, int opening, double theta, double alpha,
                       const int64_t *sel, int64_t nsel, double *acc, uint32_t *npp,
                       uint32_t *npn, double *pot, int keep_lists, int nthreads);
int ora_tree_get_lists(const ora_tree *t, int64_t nsel, int64_t *off, int64_t *list);
int ora_direct(const double *pos, const double *mass, int64_t n, const ora_params *p,
               const int64_t *targets, int64_t ntargets, double *acc, int nthreads);
int ora_direct_pot(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   const int64_t *targets, int64_t ntargets, double *acc, double *pot,
                   int nthreads);
int ora_cell_exact(const double *pos, const double *mass, int64_t n, const ora_params *p,
                   const int64_t *targets, int64_t ntargets, double *acc, int nthreads);
int ora_num_threads(void);

#endif
