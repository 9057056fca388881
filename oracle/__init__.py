"""Oracle: a plain, slow, obviously correct CPU implementation of the analyser.

TEST INFRASTRUCTURE ONLY.  The product path (``paper_2502_09202_gb300``, its CUDA
library and its Python binding) never imports, links or runs anything here.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path: the only module both
sides touch is the seeded input generator ``paper_2502_09202_gb300.synth``.

Layout
  measures.c    integer measures in plain C loops (pyramid, block search, AMM
                sum, motion-compensated sums)
  build.py      compiles measures.c with gcc into liborc.so
  measures.py   ctypes wrapper, field extraction, FP64 finalisation (NCC, SWR, AMM, ACT)
  analyser.py   the detectors (shot fast/deep check, sampling structure,
                dynamic keyframes) run sequentially over a whole clip
  dis.py        the dense sub-pixel flow estimator (inverse search per patch,
                coarse to fine, densification) in FP64 numpy

Parity status: the integer measures are pinned by closed forms, invariants and
brute force (tests/test_oracle_pins.py); the decisions are pinned by planted
ground truth of the synthetic generator.  The measure VALUES themselves are
"parity unpinned" against the paper, which prints no worked example.
"""
