"""FP64 CPU oracle for the discrete dipole approximation (DDA) hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only the tests, the smoke check and the CPU baseline
leg of the benchmark use it.  It shares no code with the CUDA library (no
kernels, headers, tables or helpers); the only common module is the seeded
workload description, which holds no arithmetic of the method.

Everything here is a plain, slow, obviously correct restatement of the method
described in the DDSCAT 7.1 User Guide (Draine & Flatau 2010) and the papers
it delegates the formulas to:

  targets.py        lattice targets (guide, "Target Generation")
  orientation.py    target orientation and incident beam (guide, "Target
                    Orientation", "Incident Polarization State")
  polarizability.py Clausius-Mossotti / LATTDR / GKDLDR (guide, "Dipole
                    Polarizabilities"; Draine & Goodman 1993; Gutkowicz-Krusin &
                    Draine 2004)
  interaction.py    the matrix A of A P = E (guide, eq. AP=E; Draine 1988),
                    direct O(N^2) product, dense matrix, and the zero-padded FFT
                    convolution (Goodman, Draine & Flatau 1991)
  solvers.py        dense LU, BiCGstab (van der Vorst 1992), CCG (CG on the
                    normal equations, Petravic & Kuo-Petravic 1979)
  observables.py    Q_ext, Q_abs, Q_sca, Q_pha, f_ml, S_1..S_4, Mueller S_ij,
                    the angular quadrature for <cos>, Q_sca (guide, "Scattering
                    Amplitude Matrix", "Mueller Matrix", "Averaging over
                    Scattering Directions")
  mie.py            Mie series for a homogeneous sphere (Bohren & Huffman 1983,
                    ch. 4)
  unet.py           FP64 reference 3-D convolution / pooling / upsampling and
                    their gradients for the learned warm start
  dda.py            end-to-end driver used by the tests

Units: lattice spacing d = 1, Gaussian units, time dependence exp(-i omega t),
incident amplitude |E0| = 1.
"""
