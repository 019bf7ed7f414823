"""FP64 CPU oracle for batched rigid-body kinematics and dynamics.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package. The CUDA
product path never calls it, and it shares no code with that path (it reads
models and states from ``gen`` like every other caller).

What it computes, and what fixes each result:

* ``rbd.fk``, ``rbd.jacobian``   forward kinematics ^0T_i(q) and frame
  Jacobians (Sec. II; Table III notation).
* ``rbd.rnea``                   inverse dynamics, Eq. 1 with f = 0, by the
  recursive Newton-Euler algorithm of Featherstone's formulation (Sec. II).
* ``rbd.crba``                   the joint-space mass matrix M(q) by the
  composite-rigid-body algorithm (Sec. II).
* ``rbd.ltdl``                   the unique factorisation M = L^T D L with L
  unit lower triangular (the Cholesky-style solve the paper recommends in its
  Sec. VI footnote), written as its plain definition via a dense Cholesky of
  the index-reversed matrix.
* ``rbd.aba``                    forward dynamics as Eq. 2 itself:
  qdd = M^-1 (tau - c - g), a dense solve. ``rbd.aba_recursive`` is the
  articulated-body recursion, kept as a second formulation for tests.
* ``mask_form``                  the paper's Algorithm 1 (vectorized RNEA) and
  Algorithm 2 (vectorized CRBA) with the ancestor mask U (Sec. III), a second,
  independent formulation of RNEA and CRBA.
* ``derivatives``                exact derivatives of RNEA and of forward
  dynamics by complex-step differentiation (step 1e-30), and the
  vector-Jacobian products built from them.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms
(single and double pendulum, a single free rigid body), invariants (M SPD,
columns of M from RNEA, kinetic energy, power balance, the skew property),
Lagrangian brute force and finite differences. No function is "parity
unpinned".

Conventions (readings of the paper where it is silent):
spatial vectors are [angular; linear] (Featherstone); body frames sit after
their joint, ^lambda T_i = placement_i * joint_i(q_i); gravity enters as the
fictitious base acceleration a_0 = [0; -g]; a free-flyer root has
q = [p (3), quat (x, y, z, w)] and qd = body-frame twist [w_b; v_b].
"""
