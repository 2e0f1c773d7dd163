"""FP64 CPU oracle for the GridSPT hot path (arXiv:1807.04215).

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously-correct
restatement of what the GPU library computes, written from the paper:

* ``cosmology``  -- BBKS linear spectrum and its sigma_8 normalisation.
* ``rng``        -- Philox4x32-10 counter-based generator (published definition).
* ``spt``        -- Gaussian initial field, the real-space recursion (Eq.
                    ``recursion_formula``, Sec. II.B) following the GridSPT
                    recipe of Sec. II.C, with full-complex FP64 FFTs.
* ``estimators`` -- shell power spectrum (Eqs. ``pk_lin``/``pk_1loop``/
                    ``pk_2loop``) and the FFT shell bispectrum (Eq. ``bk_tree``).
* ``kernels``    -- analytic Fourier-space kernels F_n, G_n (Eq.
                    ``PT_recursion_fourier``) used only to pin the grid results.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. The GPU library shares no code with it and never
imports it; nothing here imports the GPU library.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a brute-force sum, an invariant or a published value; none is
"parity unpinned".
"""
