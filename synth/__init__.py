"""Seeded synthetic atomistic systems (inputs only; no potential arithmetic)."""
from .systems import (  # noqa: F401
    System, MASSES, config1_system, water_system, csh_system, sio2_system,
    lattice_system, molecules_system, maxwell_boltzmann, dimer_system, cluster_system,
    bench_workloads, nanoparticle_mixture_system,
)
from .models import PRESETS, NU, preset  # noqa: F401,E402
