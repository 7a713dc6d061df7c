"""FP64 CPU oracle for the finite-difference micromagnetic hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything under ``oracle/``; only the test-suite, the package smoke
check and the CPU-baseline leg of the benchmark do.  The oracle is a plain,
slow, obviously-correct restatement of the equations of arXiv 2302.08843
(magnum.np) in float64 NumPy (plus one plain C brute-force sum), written
independently of the CUDA implementation: the two share no code.

Array convention: the paper's own, ``(nx, ny, nz)`` for scalar fields and
``(nx, ny, nz, 3)`` for vector fields (Sec. 2, "Design": one value per cell,
stored as a (nx, ny, nz, c) tensor).

Modules
-------
constants : mu0 and the reduced gyromagnetic ratio (Eq. llg).
newell    : Newell f/g functions, the six cell-averaged demag tensor
            components, the dipole far field (Eq. dipole), and the assembled
            tensor over all cell offsets (Sec. 4.4).
demag     : demag field as the plain direct sum (Sec. 4.4, discrete
            convolution) and as a zero-padded FFT convolution.
fields    : exchange (Sec. 4.2), uniaxial anisotropy (Sec. 4.1), Zeeman,
            energies (Eq. linear_energy_discrete).
llg       : LLG right-hand side (Eq. llg), classic RK4, Dormand-Prince 5(4),
            renormalisation, relaxation (Sec. 3).
adjoint   : hand-derived discrete adjoint of one RK4 step (Sec. 5.2 uses
            autograd for the same gradient).

Parity status: every function here is pinned by tests in ``tests/``
(closed forms, invariants, brute force) except where a docstring says
"parity unpinned".
"""
