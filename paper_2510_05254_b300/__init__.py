"""B300 (sm_103a) implementation of the nodal discontinuous Galerkin + explicit Runge-Kutta hot
path of arXiv:2510.05254: the DG right-hand side fused with the RK stage update, for linear
advection and isothermal Euler in 1D/2D/3D on LGL elements of degree 1..7.

All computation is in libndg.so (hand-written CUDA behind the C ABI of include/ndg.h); the Python
modules only marshal arguments:

  native   ctypes binding with the C names (ndg_create_ex, ndg_set_state, ndg_step, ndg_norms,
           ndg_batch_*, ndg_partition_*, ndg_pool_*, ...); loads the in-tree library;
  solver   Solver (one context: set_state / step / norms / get_state / autotune) and Batch;
  serving  the arrival driver of the serving pool (Poisson submissions, latency statistics);
  studies  the convergence and efficiency studies of the paper's Sec. 3.1 on the GPU path;
  inputs   seeded synthetic initial conditions (no method arithmetic);
  build    compiles csrc/ with nvcc for sm_103a into libndg.so.

    from paper_2510_05254_b300.solver import Solver
    s = Solver(2, 7, (256, 256), velocity=(1.0, 0.5, 0.0), dtype="f64")   # or "f32", "f64ff"
    s.set_state(U0)                        # numpy or CUDA tensor, shape (nvar, nelem, n^dim)
    s.step(s.stable_dt(0.1), 1000, 4)      # RK4; 3 and 6 also
    print(s.norms())
"""
