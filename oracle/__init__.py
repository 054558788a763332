"""Independent CPU oracle for the encrypted FFConv layer (RNS-BFV, coefficient domain).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
reference legs may import this package.  It shares no code, header, table or constant
generator with the CUDA library under paper_2102_03494_gb300/, and never imports it.

Modules:
  ring     exact Z_q / Z_q[X]/(X^N+1) arithmetic (C, 128-bit products, '%' reduction)
  params   primes, roots, CRT constants (readings of BFV's unstated parameters)
  prng     SplitMix64 counter-based draws; ternary, uniform and Gaussian samplers
  encoder  slot encoder/decoder (t = 1 mod 2N)
  bfv      keys, encryption, decryption, key switching, rotations, MulPC, AddCC, rescale
  ffconv   plain factorized convolution (Eq. 1, Eq. 2) and the encrypted layer (Sec. 4.2)

Parity status of each part is recorded in the module docstrings and in the design notes:
the ring, encoder, decryption and the layer's decrypted output are pinned by closed forms
and library routines; ciphertext bits of key switching are pinned only through decryption
identities (the paper fixes no key-switching algorithm).
"""
