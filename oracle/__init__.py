"""CPU oracle for the homomorphic convolution of "Hyena" (arXiv 2311.12519).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the paper's method, written before and independently of the
CUDA library.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
reference legs of bench.py may import, call, link or execute anything here;
the product path (paper_2311_12519_gb300) never does, and the oracle never
imports the product package.  The two share no code; only the seeded
workload generators in synth/ (which hold none of the method's arithmetic)
feed both.

Layout:
  params.py       Sec. 3.2.1 parameter selection (primes, h_{p,n}, k)
  hyena_oracle.c  ring arithmetic: NTT (natural order), negacyclic product,
                  automorphism, samplers, encryption, Galois keys, hoisted
                  key switching, CMult/PMult -- every product is a 128-bit
                  multiply followed by `%`
  bfv.py          Sec. 2.3 BFV operations on top of the C core
  conv.py         the plain convolution definition, the slot layout and the
                  Hyena layer of Sec. 3.1 with eager reduction

Pins (tests/test_oracle_*.py, all `-m "not gpu"`): the paper's worked
example (n = 2048, p = 307201 -> h = 84248, k = 11), the closed form
h^2 = -1/2 (mod p), schoolbook negacyclic products, direct DFT evaluation,
published SplitMix64 outputs, decrypt(encrypt(m)) = m, rotation of slots,
the Hadamard identity of Eq. 1, and decrypt(layer) = (2k) conv mod t
against torch's conv2d.
"""
