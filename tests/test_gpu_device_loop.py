"""The residual stopping rule run on the device (the solve loop inside the cluster
kernels for small periodic lattices, a CUDA graph with a conditional WHILE node for the
others) against the same rule evaluated on the host from fixed-step runs.

Rule: after a chunk that ends at sweep t, stop when max|f_C(t) - f_C(t-1)| / max|f_C(t)|
< tol.  On a periodic lattice the pull is a permutation of the entries, so the primal
rule equals max|f_S(t+1) - f_S(t)| / max|f_S(t+1)| of the streamed states the API
returns; the adjoint rule compares phi_C directly.  Checked: same stopping sweep, same
state bit for bit, same last residual.
"""
import numpy as np
import pytest

from paper_2609_31347_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda")


@pytest.fixture(scope="module")
def lbm_mod():
    from paper_2609_31347_b300 import lbm
    assert torch.cuda.is_available()
    lbm.load_library()
    return lbm


def rel_change(a, b):
    return np.abs(a - b).max() / np.abs(a).max()


def host_rule(s, which, run, check_every, tol, max_steps, carry=False):
    """Steps and last residual of the rule evaluated on the host from fixed-step runs:
    chunks of check_every sweeps, the residual after t sweeps from the states of sweeps
    t and t - 1 (populations `which` of the API).  An adjoint solve starts from rest
    unless phi_C was set since the last one, so with `carry` each run continues from
    the state the previous one left."""
    steps, r, last = 0, None, None

    def step(k):
        nonlocal last
        if carry and last is not None:
            s.set_populations(which, last)
        run(k, fixed_steps=True)
        last = s.get_populations(which)
        return last.cpu().numpy()

    while steps < max_steps:
        prev = step(check_every - 1)
        cur = step(1)
        steps += check_every
        r = rel_change(cur, prev)
        if r < tol:
            break
    return steps, r


# 32^2: cluster kernel through L2; 64^2: lattice in distributed shared memory;
# 130 x 67: graph-replayed sweeps under a conditional WHILE node
@pytest.mark.parametrize("kernel", ["fp64", "auto"])
@pytest.mark.parametrize("nx,ny,tol", [(32, 32, 1e-9), (64, 64, 1e-8), (130, 67, 1e-6)])
def test_device_loop_matches_the_host_rule(lbm_mod, nx, ny, tol, kernel):
    F = I.fourier_force(nx, ny=ny, seed=3, kmax=2)
    dstar = I.fourier_force(nx, ny=ny, seed=4, kmax=3) * 1e-3
    E, nu, ce = 1.0, 0.3, 64
    mk = lambda: lbm_mod.LBMSolid(nx, ny, 1.0 / nx, E, nu, control="force_field",  # noqa: E731
                                  kernel=kernel)
    a, b = mk(), mk()
    for s in (a, b):
        s.set_target(dev(dstar))
        s.set_control(dev(F))
    max_steps = 400 * nx * ny // 8 + 4000
    # primal: the first chunk starts with the collide-only sweep from rest on both sides
    info = a.primal_solve(max_steps, tol=tol, criterion=1, check_every=ce)
    # host side: f_S(t) and f_S(t - 1) in the API's streamed form
    steps, r = host_rule(b, 0, b.primal_solve, ce, tol, max_steps)
    assert info.steps == steps
    assert np.array_equal(a.get_populations(0).cpu().numpy(), b.get_populations(0).cpu().numpy())
    assert abs(info.last_metric - r) <= 1e-12 * r
    # adjoint from rest (its first sweep writes -j)
    a.objective()
    b.objective()
    info = a.adjoint_solve(max_steps, tol=tol, criterion=1, check_every=ce)
    steps, r = host_rule(b, 2, b.adjoint_solve, ce, tol, max_steps, carry=True)
    assert info.steps == steps
    assert np.array_equal(a.get_populations(2).cpu().numpy(), b.get_populations(2).cpu().numpy())
    assert abs(info.last_metric - r) <= 1e-12 * r
    a.close()
    b.close()
