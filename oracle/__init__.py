"""Oracle: a plain, slow, FP64 CPU statement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2412_09734_gb300``) and neither imports the other.

Modules
  pdhg   -- scaling (Ruiz, Pock-Chambolle), power iteration, the PDHG steps of
            eqs. (3), (5), (6), Halpern with reflection (eq. 4), r^2HPDHG
            (Algorithm 1), rAPDHG (Algorithm 2), the relative KKT error.
  brute  -- brute-force checkers that pin the converged answers: LP vertex
            enumeration and QP active-set enumeration on tiny instances.
  adjoint -- LP optimal-value gradients and the QP active-set implicit adjoint.
  unrolled -- gradients of a QP solve by differentiating through its rAPDHG
            steps along the path it took (reverse sweep over the taped path).
  spo    -- the SPO+ surrogate loss and its subgradient.
"""
