"""GB300-native cutoff non-bonded force path (LJ 12-6 + cutoff Coulomb over a periodic
cell list) with velocity-Verlet integration, behind a C ABI of hand-written sm_103a
CUDA kernels.  ``api`` is the thin binding; ``workloads`` holds the seeded inputs."""
