"""CPU oracle for noisy-shot sampling of cultivation-shaped Clifford+T circuits.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python binding)
imports, links or runs this package; only the tests, the smoke check and the benchmark's CPU
baseline leg do.  It shares no code with the CUDA path: the circuit parser, the counter-based
random number generator, the fault sampler, the stabiliser analysis, the frame pre-screen and the
simulators here are written separately from the paper's description, in plain NumPy and FP64.

Modules (each function cites the passage of the paper it follows):
  circuit     text format parser, noise-channel and readout enumeration
  philox      Philox4x32-10 and the random-number contract (fault draws, readout uniforms)
  statevector FP64 state-vector simulator, the plain definition of a shot (Sec. 4)
  mps         FP64 matrix-product-state simulator with the written truncation rule (Sec. 3.1)
  tableau     CHP stabiliser tableau (Aaronson & Gottesman) used to pin the simulators
  prescreen   offline stabiliser tracking and the per-shot Pauli pre-screen (Sec. 4.2), with the
              GF(2) sensitivity-matrix route as an independent second computation
  stats       subset-sampling reweighting, estimators, intervals, loss factor (Sec. 4.1, App. C, D)
  sampler     the per-shot pipeline producing per-weight counts
"""
