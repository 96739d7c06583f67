"""CPU oracle for the ASCC amplitude-residual hot path (test infrastructure).

Plain, slow, FP64 NumPy code written from the paper (arXiv 2501.10515,
"Improving Aufbau Suppressed Coupled Cluster Through Perturbative Analysis").
It is test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  It shares no code with the CUDA path
and never imports it.

Modules
  hamiltonian   bare Hamiltonian from (eps, B); similarity transform
                H-bar = exp(S^+) H exp(-S^+) (Eq. sim); T1 dressing.
  amplitudes    amplitude layouts, the P/M/N partition (Eq. pnm split), the
                mixed-triples slice T3' (Sec. II.B.1), the initial guess
                (Eq. TP-guess) and the spin relations (Eqs. S1-S2).
  bruteforce    O-BF: determinant-space definition of the projected
                equations (Eqs. energy, amp) and FCI.
  spinorb       O-SO: spin-orbital factorised residual.
  spinadapted   O-SA: spin-adapted closed-shell residual (the hot-path oracle).
  solver        diagonal-Jacobian update with DIIS (Sec. III.B).
  twocsf        two-CSF ASCC (Sec. II.B.2) by brute force: reference, guess,
                T3'/T4'/T5' slices, Newton solve (tiny systems only).
"""
