"""Seed bookkeeping shared by every consumer of the synthetic inputs."""

def random_pair_amplitude_seed(n_pairs, tag=0):
    """Deterministic seed for random test amplitudes of a system with n_pairs."""
    return 1234 + 7919 * int(n_pairs) + 104729 * int(tag)
