// Formulations as 2x2 block operators over {M, V, K, T, D} x {Laplace, Yukawa}
// (paper, "Boundary integral formulations"). Galerkin form: the identity
// becomes the mass matrix M, each boundary operator its weak form.
#include <string.h>

#include "internal.h"

namespace pb {

namespace {

// one block row: coefficients acting on u (col 0) and on v (col 1)
struct Row {
    double u[O_N];
    double v[O_N];
};

Row zero_row() {
    Row r;
    memset(&r, 0, sizeof(r));
    return r;
}

Row add(const Row& a, double s, const Row& b) {
    Row r;
    for (int o = 0; o < O_N; ++o) {
        r.u[o] = a.u[o] + s * b.u[o];
        r.v[o] = a.v[o] + s * b.v[o];
    }
    return r;
}

Row scale(double s, const Row& a) { return add(zero_row(), s, a); }

// interior system in interior unknowns (paper eq. bie:int:int):
//   [1/2 I + K_int, -V_int; -D_int, 1/2 I - T_int]
void int_int(Row& r1, Row& r2) {
    r1 = zero_row(); r2 = zero_row();
    r1.u[O_M] = 0.5; r1.u[O_KL] = 1.0; r1.v[O_VL] = -1.0;
    r2.u[O_DL] = -1.0; r2.v[O_M] = 0.5; r2.v[O_TL] = -1.0;
}
// exterior system in interior unknowns (paper eq. bie:ext:int), r = eps_int/eps_ext:
//   [1/2 I - K_ext, r V_ext; D_ext / r, 1/2 I + T_ext]
void ext_int(double r, Row& r1, Row& r2) {
    r1 = zero_row(); r2 = zero_row();
    r1.u[O_M] = 0.5; r1.u[O_KY] = -1.0; r1.v[O_VY] = r;
    r2.u[O_DY] = 1.0 / r; r2.v[O_M] = 0.5; r2.v[O_TY] = 1.0;
}
// exterior system in exterior unknowns (paper eq. bie:ext:ext):
//   [1/2 I - K_ext, V_ext; D_ext, 1/2 I + T_ext]
void ext_ext(Row& r1, Row& r2) {
    r1 = zero_row(); r2 = zero_row();
    r1.u[O_M] = 0.5; r1.u[O_KY] = -1.0; r1.v[O_VY] = 1.0;
    r2.u[O_DY] = 1.0; r2.v[O_M] = 0.5; r2.v[O_TY] = 1.0;
}
// interior system in exterior unknowns (paper eq. bie:int:ext):
//   [1/2 I + K_int, -V_int / r; -r D_int, 1/2 I - T_int]
void int_ext(double r, Row& r1, Row& r2) {
    r1 = zero_row(); r2 = zero_row();
    r1.u[O_M] = 0.5; r1.u[O_KL] = 1.0; r1.v[O_VL] = -1.0 / r;
    r2.u[O_DL] = -r; r2.v[O_M] = 0.5; r2.v[O_TL] = -1.0;
}

void to_blockop(const Row& r1, const Row& r2, BlockOp* B) {
    for (int o = 0; o < O_N; ++o) {
        B->c[0][0][o] = r1.u[o];
        B->c[0][1][o] = r1.v[o];
        B->c[1][0][o] = r2.u[o];
        B->c[1][1][o] = r2.v[o];
    }
}

}  // namespace

bool form_is_exterior(int form) {
    return form == PB_DIRECT_EXT || form == PB_DIRECT_EXT_PERM || form == PB_CFIE_EXT || form == PB_PMCHWT_EXT ||
           form == PB_MULLER_EXT || form == PB_LU;
}

// alpha, beta and the scale of row 2 of the CFIE family members
static int cfie_params(int form, double r, double alpha, double beta, double* a, double* b, double* s2) {
    *s2 = 1.0;
    switch (form) {
        case PB_CFIE_INT: case PB_CFIE_EXT: *a = alpha; *b = beta; return PB_OK;
        case PB_PMCHWT_INT: case PB_PMCHWT_EXT: *a = -1.0; *b = -1.0; return PB_OK;
        case PB_MULLER_INT: case PB_MULLER_EXT: *a = 1.0; *b = 1.0; return PB_OK;
        case PB_JUFFER: *a = 1.0 / r; *b = r; return PB_OK;  // alpha = eps_ext/eps_int, beta = eps_int/eps_ext
        case PB_LU: *a = r; *b = 1.0 / r; *s2 = r; return PB_OK;
        default: return set_error(PB_EINVAL, "unknown formulation %d", form);
    }
}

static int check_params(const pb_params* prm) {
    if (!prm) return set_error(PB_EINVAL, "NULL pb_params");
    if (!(prm->eps_int > 0.0) || !(prm->eps_ext > 0.0) || !(prm->kappa >= 0.0))
        return set_error(PB_EINVAL, "need eps_int > 0, eps_ext > 0, kappa >= 0");
    return PB_OK;
}

int system_blockop(const pb_params* prm, int form, double alpha, double beta, BlockOp* B) {
    PB_TRY(check_params(prm));
    const double r = prm->eps_int / prm->eps_ext;
    Row i1, i2, e1, e2, r1, r2;
    switch (form) {
        case PB_DIRECT_INT: case PB_DIRECT_INT_PERM:  // paper eq. bie:dirichlet:int
            int_int(i1, i2); ext_int(r, e1, e2);
            r1 = i1; r2 = e1;
            break;
        case PB_DIRECT_EXT: case PB_DIRECT_EXT_PERM:  // paper eq. bie:dirichlet:ext
            ext_ext(e1, e2); int_ext(r, i1, i2);
            r1 = e1; r2 = i1;
            break;
        case PB_CFIE_INT: case PB_PMCHWT_INT: case PB_MULLER_INT: case PB_JUFFER: {
            double a, b, s2;  // paper eq. bie:combined:int
            PB_TRY(cfie_params(form, r, alpha, beta, &a, &b, &s2));
            int_int(i1, i2); ext_int(r, e1, e2);
            r1 = add(i1, a, e1);
            r2 = add(i2, b, e2);
            if (form == PB_PMCHWT_INT) { r1 = scale(-1.0, r1); r2 = scale(-1.0, r2); }  // printed sign
            break;
        }
        case PB_CFIE_EXT: case PB_PMCHWT_EXT: case PB_MULLER_EXT: case PB_LU: {
            double a, b, s2;  // paper eq. bie:combined:ext
            PB_TRY(cfie_params(form, r, alpha, beta, &a, &b, &s2));
            ext_ext(e1, e2); int_ext(r, i1, i2);
            r1 = add(e1, a, i1);
            r2 = scale(s2, add(e2, b, i2));
            break;
        }
        default: return set_error(PB_EINVAL, "unknown formulation %d", form);
    }
    if (form == PB_DIRECT_INT_PERM || form == PB_DIRECT_EXT_PERM) to_blockop(r2, r1, B);
    else to_blockop(r1, r2, B);
    return PB_OK;
}

// right-hand side rows: rhs_row = d * b_D + n * b_N
int rhs_coefs(const pb_params* prm, int form, double alpha, double beta, double d[2], double n[2]) {
    PB_TRY(check_params(prm));
    const double r = prm->eps_int / prm->eps_ext;
    d[0] = d[1] = n[0] = n[1] = 0.0;
    switch (form) {
        case PB_DIRECT_INT: d[0] = 1.0; break;
        case PB_DIRECT_INT_PERM: d[1] = 1.0; break;
        case PB_DIRECT_EXT: d[1] = 1.0; break;
        case PB_DIRECT_EXT_PERM: d[0] = 1.0; break;
        case PB_CFIE_INT: case PB_MULLER_INT: case PB_JUFFER: d[0] = 1.0; n[1] = 1.0; break;
        case PB_PMCHWT_INT: d[0] = -1.0; n[1] = -1.0; break;
        case PB_CFIE_EXT: case PB_PMCHWT_EXT: case PB_MULLER_EXT: case PB_LU: {
            double a, b, s2;  // diag(alpha, beta) [phi_D; r phi_N], row 2 scaled for Lu
            PB_TRY(cfie_params(form, r, alpha, beta, &a, &b, &s2));
            d[0] = a;
            n[1] = s2 * b * r;
            break;
        }
        default: return set_error(PB_EINVAL, "unknown formulation %d", form);
    }
    return PB_OK;
}

// Calderon operators of the PMCHWT forms (paper eqs. prec:calderon:int, prec:calderon:ext)
int calderon_blockop(const pb_params* prm, int form, int which, BlockOp* B) {
    PB_TRY(check_params(prm));
    const double r = prm->eps_int / prm->eps_ext;
    Row r1 = zero_row(), r2 = zero_row();
    bool lap;
    double sv, sd;  // scale of V and of D
    if (form == PB_PMCHWT_INT) {
        lap = which == 0;
        sv = lap ? 1.0 : r;
        sd = lap ? 1.0 : 1.0 / r;
    } else if (form == PB_PMCHWT_EXT) {
        lap = which == 0;
        sv = lap ? 1.0 / r : 1.0;
        sd = lap ? r : 1.0;
    } else {
        return set_error(PB_EINVAL, "Calderon preconditioning needs a PMCHWT formulation");
    }
    r1.u[lap ? O_KL : O_KY] = -1.0;
    r1.v[lap ? O_VL : O_VY] = sv;
    r2.u[lap ? O_DL : O_DY] = sd;
    r2.v[lap ? O_TL : O_TY] = 1.0;
    to_blockop(r1, r2, B);
    return PB_OK;
}

// (a, b) of the scaled mass on top of a half Calderon preconditioner: the
// accumulation points 1/4 + eps_ext/(4 eps_int) and 1/4 + eps_int/(4 eps_ext)
// (paper eq. precond:calderon:eigenval_semi), in the order of the blocks they
// land on.
int half_calderon_scaling(const pb_params* prm, int form, int which, double* a, double* b) {
    double l1 = 0.25 + prm->eps_ext / (4.0 * prm->eps_int);
    double l2 = 0.25 + prm->eps_int / (4.0 * prm->eps_ext);
    bool first = (form == PB_PMCHWT_INT && which == 0) || (form == PB_PMCHWT_EXT && which == 0);
    *a = first ? l1 : l2;
    *b = first ? l2 : l1;
    return PB_OK;
}

}  // namespace pb
