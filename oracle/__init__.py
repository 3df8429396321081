"""CPU oracle for the mixed-precision Wilson-Dirac solver (test infrastructure only).

Plain, slow, float64 restatement of what the paper's method computes:

* ``gamma``   -- Dirac matrices in the representation fixed by the printed
                 (1 - gamma_1) of Eq. 2 (Sec. 2).
* ``wilson``  -- the Wilson matrix D_W of Eq. 1 built from explicit 4x4 spin
                 matrices and 3x3 links (no spin projection), the even-odd
                 Schur operator and source/reconstruction of Eqs. 4-6, and
                 dense assembly for tiny lattices.
* ``solvers`` -- textbook BiCGStab, the refinement loops of Algorithms 2-3 and
                 the rescaled BiCGStab of Algorithms 4-5 with emulated
                 low-precision storage.
* ``ptc``     -- the learned parallel-transport preconditioner (forward,
                 adjoint and weight gradient) in float64.
* ``clover``  -- the clover term and the even-odd system with clover blocks.
* ``arith16`` -- the hopping term evaluated in FP16 arithmetic (every
                 operation rounded to FP16), the paper's _Float16 build,
                 emulated in float64 in an order of evaluation read as the
                 kernel's.
* ``flops``   -- the hop in Sec. 2's three steps on numbers that count their
                 own real operations (the 168 flops per hop).

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference leg may import it. It shares no
code with the CUDA library; both consume inputs from
``paper_2602_14450_gb300.synth`` only.
"""
