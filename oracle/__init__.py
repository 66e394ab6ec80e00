"""CPU oracle for the Spiking Neural Dedispersion (SND) hot path (arXiv 2606.15361).

TEST INFRASTRUCTURE ONLY. This package is plain, slow, obviously-correct numpy
(FP64 wherever floating point appears). Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm may import it. The product path
(the C-ABI library and its Python binding) never imports, links or executes it,
and shares no code, header, table or constant generator with it.

Modules and the passages they follow:

* ``delays``     - cold-plasma delay and integer per-channel delay (Methods,
                   "Incoherent dedispersion").
* ``encoder``    - two-pass sigma clip and the delta encoder (Methods, "Input
                   encoding", Eq. for x_c(t)).
* ``tree``       - SND leaf clusters, B-ary levels and the three activation modes
                   (Methods, "The Spiking Neural Dedispersion algorithm"), plus
                   direct brute-force dedispersion (Methods, "The neuromorphic
                   dedispersion neuron").
* ``mf``         - DM-scaled boxcar matched filter (Methods, "Matched filtering").
* ``candidates`` - thresholding, 9x9 binary closing, 8-connected labelling and
                   peak selection (Methods, "Candidate detection").
* ``stream``     - chunked streaming with emitted-sample bookkeeping (Methods,
                   "Pipeline overview").
* ``analytic``   - closed forms used as pins: fire probability, the cascade
                   recursion (Eq. cascade) and SNR_A (Eq. snr_A).
* ``cxx``        - the same definitions once more in plain C++17 with OpenMP over
                   trial-DM rows (``cpp/snd_oracle.cpp``), fast enough to check the
                   full 1024-channel / 2048-DM stream cell by cell; pinned to the
                   modules above and to the paper's invariants.

Where the paper is silent or ambiguous, each function states the reading it
takes. Nothing here is "parity unpinned" except the candidate identity beyond the closing/labelling pins
(no printed values exist for it), which the candidates module header says.
"""
from . import analytic, candidates, delays, encoder, mf, stream, tree  # noqa: F401
