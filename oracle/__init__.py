"""CPU oracle for chordally decomposed ADMM (Zheng, Fantuzzi, Papachristodoulou, Goulart, Wynn,
"Fast ADMM for Semidefinite Programs with Chordal Sparsity", Sections II-IV).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never imports, links or calls it, and it shares
no code with the CUDA path.
"""

from .chordal_admm import (  # noqa: F401
    ChordalSDP,
    OracleError,
    proj_psd,
    proj_soc,
    proj_cone,
    admm_init,
    primal_iteration,
    dual_iteration,
    admm_solve,
)
