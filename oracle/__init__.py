"""FP64 CPU oracle for the layered-medium elastic multiple-scattering mat-vec.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference leg of
`bench.py` use it.  It shares no code with the CUDA library (no kernels, headers,
tables or constants); the only common input is the seeded generator module
`synthetic`, which holds none of the method's arithmetic.

Everything here is plain, slow and direct: numpy complex128 arithmetic, scipy's
Bessel/Hankel routines as library primitives, direct O(M^2) Graf sums, and the
separable Sommerfeld quadrature sums written exactly as the paper states them.

Modules and the passages they follow
------------------------------------
media       wavenumbers kp = w/sqrt(lam+2mu), ks = w/sqrt(mu)          (Sec. 2)
waves       cylindrical waves u_n, v_n, Cartesian derivatives and traction  (Sec. 2 tracdef, Sec. 4.1)
disc        closed-form disc scattering matrix per mode, rigid and traction-free (Sec. 4.1, Sec. 4.3 projection matrix)
graf        M2L translation T^{ml} by Graf's addition theorem          (Sec. 4.2)
sommerfeld  contour, branch of sqrt(xi^2-k^2), M2S (pts1/sed1/sed2), S2L (Jacobi-Anger, stm/c1/c2),
            2x2 interface reflection by the plane-wave route and by the paper's A_xi route (Sec. 3, 5.1, 5.3, 5.4, 7.3)
            and the same contour integral by adaptive Gauss-Kronrod quadrature (Sec. 5.1, reading A5)
system      mat-vec y = gamma - S (T + R) gamma, plane-wave right-hand side, GMRES, dense LU,
            receiver fields, boundary-condition residual                    (Sec. 4.2 mul2, Sec. 5.2 aequ/Schur, Sec. 7.3 bplan)
nystrom     Nystrom boundary integral solve of one star-shaped particle (Kress log and Hilbert-transform
            product quadrature), its scattering matrix by the projection formula and by the single-layer
            coefficient formula, rotated copies                               (Sec. 4.3 bdint, S7, S10; Sec. 7 shapes)
layered_bie brute-force boundary integral solve of a few particles with the layered Green's function
            (free-space part plus its Sommerfeld reflection), no scattering matrices (Sec. 7.1 direct method)
adjoint     adjoint gradient of a receiver misfit in centres, radii and omega (inverse scattering, Sec. 7.5)
sph3d       3D: spherical harmonics (continued to complex directions), vector spherical wave functions L, M, N,
            closed-form rigid and traction-free sphere scattering matrices, the plane-wave coefficients a, b, c,
            and the free-space translation by projection on a sphere about the target      (Sec. 6, 6.3)
layered3d   3D layered operator: polar Sommerfeld rule, the spectral field of a particle (block B), the
            P/SV/SH reflection at the interface, the plane-wave expansion about a particle (block C), the
            mat-vec, plane waves from the upper layer, dense solve and fields               (Sec. 6.1-6.3)

Pins (tests/test_oracle_*.py, all `-m "not gpu"`) tie each function to something other
than itself: Bessel and Hankel values against mpmath, Graf pointwise evaluation, the
Sommerfeld identities as quadrature, Jacobi-Anger on contour nodes, boundary-condition
residuals of the disc matrices, two independent derivations of the reflection matrix,
identical-media zero reflection, plane-wave energy balance for incidence from below and
above, textbook normal-incidence coefficients, interface continuity of the assembled field,
elastodynamic reciprocity of the layered field, boundary-condition residuals of the solved
multi-particle system, a manufactured solution from point sources inside the particles, a
dense-LU solve, and central differences of the loss for the adjoint gradient.  For the
non-circular particles (tests/test_oracle_nystrom.py): exactness of the product-quadrature weights
on trigonometric polynomials, the traction kernel against differences of the fundamental solution,
the Nystrom matrix on a disc against the closed form, an exact exterior solution from point forces
inside a star, S7 against S10, the solver on a rotated boundary against the rotation phase, the
multiple-scattering solve against the brute-force layered boundary integral solve of three stars,
and the fixed contour rule against adaptive Gauss-Kronrod quadrature.  For 3D (tests/test_oracle_3d.py):
orthonormality and the addition theorem of the harmonics, differences of the harmonics and of the wave
functions' curls, the exponential itself for the plane-wave coefficients at real and complex
directions, sphere boundary conditions, the local expansion reproducing the sources' field, the projection
translation against the scalar addition-theorem series written out with Gaunt integrals, the polar
quadrature of the spectral representation reproducing the outgoing field, zero reflection between
identical layers, energy balance, and the solved system's boundary residual falling with the order.
"""
