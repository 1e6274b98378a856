"""CPU FP64 oracle for the batched Helmholtz solve path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import anything from this package.
The product path (the CUDA library and its Python binding) never imports,
links or executes it, and this package imports nothing from the product.

Each function is a plain, slow, obviously-correct statement of what the
paper defines, in float64/complex128, citing the passage it follows:

* ``helmholtz``  - the discrete operator H(m, w) of Eq. 3.1-3.2 with the
  absorbing layer gamma, the shifted Laplacian of Eq. 3.12, the direct
  (sparse LU) solve that defines the answer, residual norms.
* ``multigrid``  - the shifted-Laplacian V-cycle of Sec. 3.4 (Eq. 3.12, 3.14).
  The paper does not specify smoother, transfers or coarsest solve; the
  readings implemented here are listed in the module header.
* ``krylov``     - flexible GMRES (the Krylov method of Sec. 3.4 and Eq. 4.3)
  and the fixed-iteration GMRES used for training data (Eq. 4.3, Alg. 2).
* ``fwi``        - the FWI data misfit (Eq. 3.5) and its adjoint-state
  gradient built on the conjugation identity of Sec. 4.3 (Eq. 4.4-4.8).
* ``green``      - the 2D free-space Green's function used as a pin.
* ``cnn``        - nested-loop reference of the encoder-solver U-Net layers
  (Fig. 1 caption, Eq. 3.13, 4.1), MSE (Eq. 4.2) and Adam.
* ``training``   - training pairs of Eq. 4.3, the data step of Alg. 2, the
  loss of Eq. 4.2 and the M_VU compositions of Eq. 3.14.

Random draws (the x ~ CN(0, 1) of Eq. 4.3, the GMRES step counts) are made by
the seeded input generators of ``paper_2405_17696_gb300.media`` and passed in
as inputs to both sides.
"""
