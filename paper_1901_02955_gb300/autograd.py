"""torch.autograd binding of the library's discrete adjoint (snap_record / snap_step_adjoint).

SnapSteps.apply(Y0, context, nsteps, ckpt_every, dt_fixed) advances a conserved state by
nsteps steps in the CUDA library and returns Y_N; its backward is the library's hand-written
adjoint of those steps (checkpointed every ckpt_every steps and recomputed in between, or,
with ckpt_every = 0, every stage input kept so that nothing is recomputed). The
forward and the adjoint both run in the library's kernels; torch only holds the tensors.
Inviscid single-domain contexts, dry or with one vapour in the x-z plane (the library returns
SNAP_ENOTSUP otherwise). The initial-state maps and functionals below are plain torch
expressions, so autograd chains the library's dJ/dY_0 to dJ/dtheta_0."""
import torch


class SnapSteps(torch.autograd.Function):
    @staticmethod
    def forward(fctx, Y0, context, nsteps, ckpt_every=20, dt_fixed=0.0):
        if not Y0.is_cuda:
            raise ValueError("SnapSteps needs a CUDA tensor")
        context.set_state(Y0.detach().contiguous())
        context.record(nsteps, ckpt_every, dt_fixed)
        YN = torch.empty_like(Y0)
        context.get_state(out=YN)
        fctx.context = context
        fctx.nsteps = nsteps
        return YN

    @staticmethod
    def backward(fctx, gYN):
        lam0 = fctx.context.step_adjoint(fctx.nsteps, gYN.contiguous())
        return lam0, None, None, None, None


def dry_state_from_theta(theta, p_cell, R_d=287.0, gamma_d=1.4, p0=1e5, velocity=None):
    """Conserved state of a dry gas with potential temperature theta[k, j, i] on the reference
    pressure p_cell[k] (the initial-state map of the warm-bubble workloads):
    rho = p / (R_d theta (p/p0)^kappa), rho e = p / (gamma_d - 1) + |m|^2 / (2 rho), with
    momenta rho u from an optional velocity[comp, k, j, i] (default: at rest)."""
    kappa = (gamma_d - 1.0) / gamma_d
    p = p_cell.reshape(-1, 1, 1).to(theta)
    rho = p / (R_d * theta * (p / p0) ** kappa)
    nmom = 3 if theta.shape[1] > 1 else 2
    if velocity is None:
        mom = [torch.zeros_like(rho)] * nmom
        ke = torch.zeros_like(rho)
    else:
        mom = [rho * velocity[c] for c in range(nmom)]
        ke = 0.5 * rho * (velocity ** 2).sum(dim=0)
    rhoe = p / (gamma_d - 1.0) + ke
    return torch.stack([rho] + mom + [rhoe])


def moist_state_from_theta(theta, p_cell, q_vapor, R_d, gamma_d, eps, sigma_v, n_cond=2,
                           p0=1e5, velocity=None):
    """Conserved state (rho_d, rho_v, n_cond condensates at 0, momenta, rho e) of air with one
    vapour of mass fraction q_vapor[k, j, i] (held fixed) at potential temperature theta on
    the reference pressure p_cell[k]: T = theta (p/p0)^kappa with the dry kappa,
    rho = p / (R_m T), R_m = (1 - q) R_d + q R_d / eps, and rho e = (c_vd rho_d + sigma_v c_vd
    rho_v) T + |m|^2 / (2 rho) (Sec. 2 with no condensate)."""
    kappa = (gamma_d - 1.0) / gamma_d
    c_vd = R_d / (gamma_d - 1.0)
    p = p_cell.reshape(-1, 1, 1).to(theta)
    T = theta * (p / p0) ** kappa
    q = q_vapor.to(theta)
    rho = p / (((1.0 - q) * R_d + q * (R_d / eps)) * T)
    rho_v = q * rho
    rho_d = rho - rho_v
    nmom = 3 if theta.shape[1] > 1 else 2
    if velocity is None:
        mom = [torch.zeros_like(rho)] * nmom
        ke = torch.zeros_like(rho)
    else:
        mom = [rho * velocity[c] for c in range(nmom)]
        ke = 0.5 * rho * (velocity ** 2).sum(dim=0)
    rhoe = (c_vd * rho_d + sigma_v * c_vd * rho_v) * T + ke
    cond = [torch.zeros_like(rho)] * n_cond
    return torch.stack([rho_d, rho_v] + cond + mom + [rhoe])


def kinetic_energy(Y, cell_volume, n_mass=1):
    """Domain kinetic energy sum |m|^2 / (2 rho) dV; the first n_mass fields are the
    densities whose sum is rho, the momenta follow them."""
    rho = Y[:n_mass].sum(dim=0)
    m2 = (Y[n_mass:-1] ** 2).sum(dim=0)
    return 0.5 * (m2 / rho).sum() * cell_volume


def column_cloud_mass(Y, dz, i, j=0, cloud_field=2):
    """Cloud mass per unit area of one column: sum over k of rho_c[k, j, i] dz."""
    return Y[cloud_field, :, j, i].sum() * dz
