"""Spectra of the preconditioned systems (paper, the eigenvalue figures of
"Performance of different formulations and preconditioners"): the dense
matrix P^-1 A is formed column by column from the library's own operator and
preconditioner applications on the GPU, and its eigenvalues by a dense
library eigensolver. For small meshes (the matrix is (2 N_v)^2)."""
import torch

from . import api


def preconditioned_matrix(ctx, mesh, near, params, form, precond, opts=None, prec=api.PB_F64):
    """Dense P^-1 A (2 N_v x 2 N_v, float64, on the mesh's device), one column per application."""
    n2 = 2 * mesh.info()["n_verts"]
    out = torch.empty((n2, n2), dtype=torch.float64, device="cuda")
    e = torch.zeros(n2, dtype=torch.float64, device="cuda")
    ax = torch.empty_like(e)
    col = torch.empty_like(e)
    a_, b_ = (opts.alpha, opts.beta) if opts is not None else (0.0, 0.0)
    for j in range(n2):
        e.zero_()
        e[j] = 1.0
        api.pb_system_apply(ctx, mesh, near, params, form, e, prec, a_, b_, y=ax)
        api.pb_precond_apply(ctx, mesh, near, params, form, precond, ax, y=col, opts=opts, prec=prec)
        out[:, j] = col
    return out


def spectrum(ctx, mesh, near, params, form, precond, opts=None, prec=api.PB_F64):
    """Eigenvalues (complex128 tensor) of P^-1 A."""
    return torch.linalg.eigvals(preconditioned_matrix(ctx, mesh, near, params, form, precond, opts, prec))
