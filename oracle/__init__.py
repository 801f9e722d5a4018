"""CPU reference ("oracle") for the QPT-assisted MPDO noisy-circuit update.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import anything in this package; the CUDA
library never calls it and has no CPU fallback.

Plain, slow, FP64 NumPy written from the paper's definitions:

  channels  - Eq. (chi), the chi -> Choi change of basis and the Choi
              eigendecomposition that yields Kraus operators (Sec. III).
  dense     - a 2^n x 2^n density-matrix simulator that applies every channel
              straight from Eq. (chi) (no Kraus operators at all); it is the
              exact definition the MPDO approximates when nothing is truncated.
  mpdo      - the MPDO of Sec. II.C/II.D: rank-4 site tensors T[l, p, n, r],
              noisy gates K_i = N_i U contracted with a new Kraus leg (Fig. 2),
              SVD truncation of the Kraus leg (Eq. svdNoise, Fig. 3a) and of the
              bond between two sites in canonical form (Fig. 3b), and the
              readouts built from the local density M = sum_n T T* (Sec. II.C).

NumPy's eigh / svd / qr serve as single steps; nothing is blocked, fused or
reordered beyond what the definitions state.
"""
