"""Plain FP64 CPU oracle for the accelerated dual proximal gradient (APG) solver of
scenario-tree stochastic MPC ("GPU-accelerated stochastic predictive control of
drinking water networks", Sampathirao, Sopasakis, Bemporad, Patrinos).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import or execute anything in this package; the
product path (the C-ABI library and its Python binding) never does, and shares no
code with it.  Everything here is written for a reader checking it against the
paper by eye: numpy in float64, the nodes of one stage processed together (the
paper's Algorithm 1 states they are independent), no other blocking or fusion.

Modules
-------
tree        parent array -> stages, children, paths (Sec. III-C)
factor      null-space elimination and factor step (App. A, App. B)
cost_update per-step vectors u_hat, e, alpha_bar, beta (App. A)
solve_step  Algorithm 1 (paper's three-term form)
prox        proximal operators of g (Sec. IV-C, App. C)
apg         iteration eq. apg-iteration with theta recursion and residuals
dual        dense dual Hessian, Jacobi scaling and Lipschitz constant on small
            trees (Sec. IV-D)
"""
from .apg import apg, theta_sequence  # noqa: F401
from .cost_update import cost_update  # noqa: F401
from .dual import dense_dual_hessian, jacobi_steps, lipschitz_dense  # noqa: F401
from .factor import factor  # noqa: F401
from .prox import prox_box, prox_dist, prox_g  # noqa: F401
from .solve_step import solve_step  # noqa: F401
from .tree import Tree  # noqa: F401
