"""Plain, slow, obviously correct FP64 CPU oracle for the reduced-space network constraint.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the bench's
CPU-baseline / reference leg may import this package.  The CUDA library never calls it and
shares no code with it; the two meet only through the seeded inputs of `synth`.

Contents and the passages they follow:
  nn.py        Eq. 3 (the MLP), the reverse-mode Jacobian of the constraint g(x,y) = y - NN(x)
               (Section 2, oracle list), and Eq. 6: the Hessian of the scalar lambda^T NN(x)
               by forward-over-reverse differentiation, plus the equivalent sum over layers.
  checks.py    Independent routes used to pin nn.py: complex step, hyper-dual numbers,
               central finite differences, closed forms.
  ipm.py       A primal-dual interior-point method for Eq. 1 whose Newton step is the KKT
               system of Eq. 2 (the paper leaves the terms alpha and beta unstated; they are
               read as IPOPT's barrier terms, Waechter & Biegler 2006).
  problems.py  The synthetic adversarial problem (a variant of Eq. 7) and the SCOPF-shaped
               batch (a variant of Eq. 8) in the form of Eq. 1.
  warmstart.py The warm-start network: forward, backward and the Adam update (Kingma & Ba).
"""
