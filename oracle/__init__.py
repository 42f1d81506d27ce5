"""Plain CPU FP64 oracle for the relativistic CD-ADC sigma product.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``. The
product (the C-ABI library and its Python binding) never imports it, and it
never imports the product: the two share no code. The only shared module is
``synthetic`` (seeded random inputs, no arithmetic of the method).

Modules
-------
``isr_series``  brute-force ISR in determinant space (pins every block order).
``integrals``   antisymmetrised integrals from Cholesky vectors (Eq. 43),
                MP amplitudes and the MP1/MP2 densities; a problem given
                with full occupied and virtual Fock blocks brought to the
                semicanonical basis (``semicanonical``).
``adc``         closed-form ADC(2), ADC(2)+x(3), ADC(3) blocks for IP and EA,
                the explicit secular matrix, matrix-free sigma and diagonal.
``davidson``    dense eigensolver and a plain Davidson for the lowest roots.
``fns``         frozen-natural-spinor density, truncation, semicanonicalisation
                and transformation of the Cholesky vectors (Eqs. 25-30).
``adc_ee``      closed-form EE-ADC blocks from Wick's theorem (term tables).
``rows``        single rows of the sigma at full size: IP/EA satellite and
                main rows, EE doubles rows.
``gradients``   Hellmann-Feynman derivatives of the roots (Eq. 10) along a
                direction of (B, eps, x), from central differences of the
                explicit matrix.
``properties``  ISR properties (Sec. 2.2): EE ground-to-excited transition
                densities, IP/EA spectroscopic amplitudes, state and
                state-to-state densities of every kind;
                ``isr_series.transition_moments_series`` and
                ``spectroscopic_series`` are their brute-force pins.
``cholesky``    one-step pivoted Cholesky decomposition of the two-electron
                integrals and the MO transformation of the vectors (Eqs. 41-42).
``ssfns``       state-specific natural spinors for EA and EE (Eqs. 31-32):
                state density of the zeroth-order intermediate states, guess
                transformation, root-specific solves, corrected energies.

Every function is written for clarity, in FP64 complex, with no blocking or
fusion beyond what the cited definition states.
"""
