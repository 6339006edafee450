"""FP64 CPU oracle for ExactSim single-source SimRank (Wang et al., arXiv:2004.03493).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or run anything in this package.  The library in ``paper_2004_03493_gb300``
never uses it and has no CPU fallback.  The two share no code; the only common
inputs come from the ``synth`` generators.

Parts (each cites the passage it follows):

* ``power``        -- O1: Power Method S = (c P^T S P) v I (Sec. 2.2, "Other
  Related Work") and the exact diagonal correction D = S - c P^T S P implied by
  the linearization (Eq. def-lsim2).
* ``pair_chain``   -- brute-force meeting probabilities of two sqrt(c)-walks
  (Eq. scwwalk) by an exact rational linear solve on graphs of <= 8 nodes; an
  independent formulation used to pin ``power``.
* ``linearization`` -- O2: the steps of Algorithm 1 in the paper's order: L,
  the l-hop PPR vectors, the sample-count allocation (Algorithm 1 and the
  pi(k)^2 scheme of Lemma 4), the diagonal estimate from walk counts
  (Algorithm 2), the reverse accumulation (Eq. sL), the bilinear identity
  (Eq. formula-ppr) and the top-k list.
* ``walks``        -- O3: the walk-pair sampler of Algorithm 2 in C (OpenMP) with a
  Philox-4x32-10 counter stream written from Salmon et al. (SC'11).
* ``exactsim``     -- the whole CPU query (Algorithm 1 with Algorithm 2).

Parity status of each function is stated in its module header.
"""
