"""FP64 CPU oracle of the leaf-scattering FDTD hot path.

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import or run anything in this package. The
CUDA library never routes through it, and it shares no code with the library.
fdtd_tmz_c and fdtd_tez_c run the TMz and TEz time loops in plain C
(tmz_loop.c, tez_loop.c, bit-identical to the numpy loops) for full-size
grids.
"""
from .fdtd_tmz import (  # noqa: F401
    C0, MU0, EPS0, ETA0, eps_sigma, lossy_coefficients, cpml_profile,
    source_waveform, IncidentLine, TMzOracle, run_rt,
)
