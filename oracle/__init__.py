"""FP64 CPU oracle for the Spectral Ewald k-space path (arXiv:1712.04718).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_1712_04718_gb300``) never imports it and has no
CPU fallback; the two share no code.

O1 -- classic Ewald sum (Sec. 1, Eq. 1.5-1.7): direct k-space sum, explicit
      real-space image sum, self term.
O1 also evaluates the real-space image sum at chosen target particles only
      (ewald_real_at), for checks of large systems on a sample.
O2 -- the SE k-space method (Sec. 3, Eq. 3.5-3.13) step by step: spread with
      direct exp, direct separable DFT, Green's-function scaling, inverse DFT,
      gather of potential and force; with forces by ik differentiation
      (Sec. 2.3: the scaled spectrum times i k per axis, inverse DFT, gather
      with the spreading window) in se_kspace_ik.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force and the paper's error estimates.
"""
from .oracle import *  # noqa: F401,F403
