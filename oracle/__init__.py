"""CPU FP64 oracle for ADAGIO -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or run anything in
this package.  The CUDA library never routes through it, and the two share no
code: no kernels, headers, helpers, tables or constant generators.  The only
thing both sides consume is the seeded input generators in
``paper_1609_05388_gb300.synth``, which hold none of the method's arithmetic.

Contents
  adagio.py  centring, covariance, exact PCA, the JL matrix from the SplitMix64
             counter generator, Algorithm 1's map, the embedding, the certified
             dimension search and the FP64 predictor network.
  cert.c     plain-C FP64 all-pairs certificate (Eq. 2 and Eq. 3 by direct
             coordinate differences), loaded through ``certificate.py``.
  mlp.py     FP64 forward / backward / Adam of the dimension predictor.

Parity unpinned: the predictor network's *accuracy* (there is no paper value
to pin it to; only its gradients are pinned, by finite differences).
"""
