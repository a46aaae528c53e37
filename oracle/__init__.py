"""CPU oracle (float64 NumPy) for the Kronecker-regression hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
execute anything in this package. The CUDA library never imports it, shares no
code with it, and fails loudly when its own extension is missing.

Modules:
  philox  - Philox4x32-10 and the 53-bit uniforms of the sampler
  kron    - leverage scores, product-distribution sampling, sampled products,
            Kronecker preconditioner, Alg. 2 Richardson, closed forms, dense QR
  tucker  - Alg. 3 (factor-row update with the Woodbury preconditioner) and
            Alg. 1 TuckerALS (exact and sampled)
"""
