"""Plain FP64 CPU oracle for the GPU-SLS hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls, links
or executes anything here: only tests/, the smoke check of __graft_entry__
and the CPU-baseline leg of bench.py may use it.  It shares no code with the
CUDA library; both take their inputs from paper_2604_07644_b300.workloads.

Every function follows the paper's statement of the operation and cites the
section/equation it implements.  Where the paper is garbled, the reading taken
is stated at the function.

Modules
    lq        augmented costs (eq. augmented_matrices / augmented_linear),
              sequential Riccati LQ solve, dense-KKT LQ solve
    scan      the paper's conditional-value-function elements and combine
              (eq. assoc_init, eq. combination_rules), reverse scans
              (sequential fold and the App. A up/down-sweep schedule)
    admm      step-by-step ADMM (Sec. IV-A) with the OSQP-style rho rule
    kkt       FP64 KKT residual of the LTV-QP (eq. sqp_qp)
    infeas    Farkas certificate of primal infeasibility from a multiplier
              direction (the classification of solves at max_iter)
    activeset brute-force active-set solve of tiny LTV-QPs
    sls       N Riccati recursions, Phi_x / Phi_u, margins, beta / tau
    mlp       2-hidden-layer ReLU MLP forward / backward / Adam
    fastsls   the FastSLS alternation (tightening, App. B duals, the loop)
    models    Dubins car and planar quadrotor (App. C, App. D), the
              linearized QP, merit, line search, SQP and RTI

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, dense linear algebra, brute force or invariants; the paper prints
no worked numeric example, so no pin comes from the paper's own numbers.
"""
