"""CPU oracle for AeroSketch: plain FP64 NumPy, written from the paper.

Test infrastructure only.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import, call or execute anything here; the
GPU product path in paper_2601_02019_gb300 never does and shares no code with it.

Modules:
  philox     - Philox4x64-10 and Box-Muller, from the published definition.
  fd         - exact Frequent Directions (Section 2.3).
  aerosketch - Algorithms 1-5 and 8 (persistent AeroSketch).
  metric     - covariance error (Section 5.1.2) and the FD bound.
  bounds     - closed forms the paper states (Corollary 1, Eq. 1).
"""
