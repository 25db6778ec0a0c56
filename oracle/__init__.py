"""FP64 CPU oracle for the lattice-Green's-function convolution.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_1601_00035_gb300``) never imports it and
shares no code with it.

Parity pins (each is a test in tests/test_oracle_*.py):
  * G(0) = -W/6 with Watson's closed form for W (App. B Bessel form)
  * L G = delta at every table entry (App. A Laplacian, Sec. 2.2)
  * |G - two-term asymptotic| shrinks like |n|^-5 (App. B expansion)
  * i_n(t) against mpmath's Bessel I at 30 digits
  * integrating-factor footnote values (Sec. 2.3): first n with
    G_E(n,0,0)/G_E(0) < 1e-10 is 7 (alpha = 0.1) and 13 (alpha = 1.0)
  * sum_n g_alpha(n) = 1, g_a * g_b = g_{a+b} (Neumann addition theorem)
  * direct sum: L(G*f) = f on the interior; single point source = shifted
    table; agreement with an independent zero-padded FFT convolution
  * mimetic identities of App. A (adjointness, D C = 0, C G = 0, L_C = -G^T G)
"""
from .oracle import *  # noqa: F401,F403
