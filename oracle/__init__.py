"""Plain, slow FP64 CPU oracle for the ET-AIM hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the timed CPU
baseline of the benchmark may import this package; the product path never calls
it and shares no code, tables or constants with it.

What it computes (each module cites the passage it follows):

* ``rwg``        RWG spatial basis on a triangle mesh (Sec. 3, Eq. 3).
* ``tbasis``     causal piecewise-polynomial interpolatory temporal basis, CPPIF
                 (Sec. 3, Eq. 3).
* ``blif``       band-limited interpolatory temporal basis (approximate prolate
                 spheroidal) and its causal extrapolation (Sec. 3, 3.1.2).
* ``quad``       triangle cubature rules.
* ``singular``   closed-form integrals of 1/R and (r'-r)/R over a triangle, used
                 for singularity extraction (Sec. 3.1 mentions singularity
                 extraction; the formulas follow Wilton et al. 1984 / Graglia 1993).
* ``efie``       envelope EFIE impedance matrices Z_m of ET-MOT (Eq. 4), the
                 excitation vector V_l from the modulated Gaussian (Eq. 1), and the
                 frequency-domain EFIE matrix used by the DC-identity pin.
* ``aim``        the ET-AIM operator of Eq. 5: moment-matching anter/interpolation,
                 grid Green-function envelopes, brute-force and FFT grid sums, and
                 the pre-corrected near-zone matrices (Sec. 4, stages i-iv).
* ``mfie``       the time-differentiated envelope MFIE and its frequency-domain form, for
                 the combined-field equation of Sec. 2.1 (CFIE).
* ``mfie_aim``   the AIM form of the MFIE operator (Sec. 4 on the CFIE's MFIE term): curl
                 test weights by moment matching, the grid kernel (DT) e^{-jkR}/R and the
                 pre-corrected near zone.
* ``march``      time marching of Eq. 4 (direct ET-MOT) and Eq. 5 (ET-AIM).
* ``blocked``    the delayed sums of the right-hand side by the multilevel blocked
                 schedule with temporal FFTs (Sec. 4, stage ii), and directly.
* ``mie``        Mie series for a PEC sphere (Sec. 5, reference [18]) and the dB-error
                 norm of Eq. 2.
* ``rcs``        bistatic RCS of a marched current envelope at one frequency
                 (Sec. 2.4): the CPPIF and BLIF spectra, the envelope and incident-pulse
                 transforms, and the directions and weights of the Eq. 2 integrals.

Readings of passages the paper leaves open are listed in the design notes; the
code states each one where it is used.
"""
