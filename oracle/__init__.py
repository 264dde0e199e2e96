"""Oracle: a plain, slow FP64 CPU restatement of the fourth-order cut-cell
multigrid method (Liu, Li, Yan, Li, Zhang).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only `tests/`, `__graft_entry__.smoke()` and
the `cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares
no code, tables or constants with the CUDA library; the one module both
sides use is the top-level `workloads` (seeded inputs only), which belongs
to neither.

Modules
  ghost       ghost-cell averages at grid-aligned walls (Sec. 4.1)
  geometry    cut cells of a box minus ellipses, Alg. 1 merging, moments
  discretize  SFV / PLG classification (Def. 4.1), PLG fits (Eq. 4.11-4.19),
              the assembled system A u = f - N g (Eq. 4.20-4.22)
  multigrid   A22 LU (Def. 5.3), block smoother (Def. 5.6), transfers
              (Eq. 5.10-5.11), V-cycle (Alg. 2), FMG (Alg. 3), two-grid
              operator (Eq. 5.12)
  norms       error norms (Eq. 6.1)

Every floating-point value is FP64.  Operators are applied through an
explicitly assembled sparse matrix so that every row can be read against
the paper.  Parity notes: the PLG lattice rule and the merge order are
readings of the paper (it cites another paper for the lattice search);
they are "parity unpinned" with respect to the paper and are pinned only
through invariants (exactness on polynomials, poisedness, volume bounds).
"""
