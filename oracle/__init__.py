"""CPU oracle for the PEXSI hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from this
package. The product library never does: it has its own pole table, its own
symbolic analysis and its own kernels, and shares no code with this package.

Contents (all FP64 / complex128, plain numpy / scipy):

* :mod:`oracle.poles`   -- Fermi-Dirac pole expansion (Eq. polerho, Eq. gammaF):
  shifts z_l and weights w^rho_l, w^E_l, w^F_l from (beta, Delta E, P).
* :mod:`oracle.dense`   -- the definitions the method reaches exactly:
  Gamma = Im sum_l w_l (H - (z_l + mu) S)^{-1} restricted to the pattern of H
  (Eq. gammapole, Eq. gammaF; Sec. II.A says the selected elements are exact),
  Tr[Gamma S] (Eq. Nmu) and the inertia count N(sigma) = #{eig(H,S) < sigma}
  (Sec. II.C, Sylvester's law of inertia).
* :mod:`oracle.sampled` -- the same definitions evaluated column by column
  with a sparse LU solve, for sizes where a dense inverse is too slow.
* :mod:`oracle.hermitian` -- complex Hermitian H and S (the k-point /
  spin-orbit variant, Sec. IV): Gamma = sum_l (w_l G_l - conj(w_l) G_l^H) / 2i
  on the pattern, and Tr[Gamma S].

Every function is pinned by tests in ``tests/test_oracle_pins.py`` (and
``tests/test_oracle_hermitian.py`` for the Hermitian variant) against
closed forms (generalised eigen-decomposition), invariants and special
cases. No function here is "parity unpinned".
"""
