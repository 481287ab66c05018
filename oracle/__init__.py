"""Plain FP64 CPU oracle of the LRDM Gateaux-derivative path (Das & Gavini,
arXiv 2211.07894).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The CUDA library
(``paper_2211_07894_gb300``) never imports it, and this package imports
nothing from the library: the two share no code.  The only module both sides
use is ``workloads`` (seeded input generators, which hold none of the method's
arithmetic).

Every function is written from the paper's equations (cited in each
docstring) as a direct, unblocked numpy/scipy computation in float64.
"""

from .lrdm_oracle import (  # noqa: F401
    System,
    fermi,
    electron_count,
    solve_mu,
    loewner,
    loewner_from_occ,
    loewner_recursive,
    lda_vx,
    lda_fx,
    poisson_symbol,
    hartree,
    density,
    perturbation_potential,
    project,
    dmu_shift,
    subspace_response,
    density_response,
    gateaux,
    lrdm_apply,
    alpha_schedule,
    lrdm_krylov_step,
    LrdmaState,
    lrdma_step,
    backward,
    total_eps_grad,
    fermi_recursive,
    KpointSystem,
    solve_mu_kpoints,
    density_kpoints,
    gateaux_kpoints,
    backward_kpoints,
)
