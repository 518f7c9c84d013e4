"""CPU oracle for the multilayer Gaussian-graph fast-summation path.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import, call, link
or execute anything in this package.  The product path (the CUDA library and
its Python binding) never touches it and shares no code, table or helper with
it; the two meet only through the seeded inputs of
`paper_2007_05239_gb300.workloads`.

Everything here is plain and slow on purpose, in float64:

* `graph`   - the definitions of Sec. 2: Gaussian weight matrix W with zero
              diagonal, degrees D = diag(W 1), L_sym = I - D^{-1/2} W D^{-1/2},
              the multilayer operator I - L_1 (Eq. I-L_1, Sec. 3) and the
              shifted power mean L_{p,delta}^p (Eq. L_p_delta_power_p).
              Direct O(n^2) sums, in C with OpenMP for large n
              (`direct_sum.c`) and numpy for small n.
* `alg1`    - Alg. 1 (NFFT-based fast summation, Sec. 4) with the two
              non-equispaced Fourier transforms done as direct sums (no
              window, no FFT of the point data), the Fourier coefficients
              b_l of Eq. K_RF from samples of the (regularised) kernel, and
              the readings of the domain scaling and of the regulariser.
* `eigen`   - dense eigenpairs (numpy eigh as the library step) and a
              textbook cyclic Jacobi solver used as a second opinion.

Parity status per function is listed in each module's header.
"""
