"""CPU parity oracle for the PairHMM forward algorithm.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The product
library and its binding never do.
"""
from .oracle import (  # noqa: F401
    build,
    q_phred,
    loglik_probs,
    forward_raw,
    loglik_phred,
    rowwise_eq7,
    batch,
    lib_path,
)
from .brute import brute_force_loglik, brute_force_sum  # noqa: F401
