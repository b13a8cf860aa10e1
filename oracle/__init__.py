"""FP64 CPU oracle for generalized sampling (Fourier samples -> boundary-corrected
Daubechies scaling-function coefficients), written from the paper "Generalized
Sampling in Julia" (Jacobsen, Nielsen, Rasmussen).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it. The CUDA library never calls it,
and it never calls the CUDA library: the two share no code.

Everything here is plain, slow and written to be checked by eye against the
paper: direct (O(MN)) evaluation of the change-of-basis matrix entries, a
textbook CGLS and a Householder-QR least-squares solve, all in float64 /
complex128. Numpy routines (matmul, roots, QR, FFT) serve as single steps.

Modules
-------
filters    Daubechies low-pass filter by spectral factorisation (App. A).
phihat     Fourier transform of the scaling function, infinite product (App. A).
boundary   Boundary scaling functions on the half line and their Fourier
           transforms (Sec. 3.3, App. A.1).
operator   Entries of T in 1D and 2D and direct products T x, T^H y
           (Sec. 4, Sec. 5, App. C).
weights    Voronoi density weights in 1D (Sec. 4.1).
solvers    CGLS and QR least squares (Sec. 2, Sec. 6.3).

Readings of the paper that are not literal (all flagged in the design notes):
the phi-hat product starts at j=1; the interior phase is exp(-2 pi i k xi/2^J);
rows are scaled by sqrt(mu); the boundary functions are the nested-support
Gram-Schmidt basis of the Cohen-Daubechies-Vial edge space, sign fixed by
h^L_{k,p+2k} > 0.

Parity unpinned: the boundary filter VALUES of Cohen-Daubechies-Vial (not
printed in the paper) -- only basis-invariant properties are pinned.
"""
