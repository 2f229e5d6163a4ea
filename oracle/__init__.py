"""CPU oracle of the Ozaki-Bailey FFT.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline and reference legs may import, link or run anything here.  The
product path (the CUDA library and its binding) never touches it, and the two
share no code: the oracle computes its constants with Python integers and its
arithmetic with plain C (ozaki_ref.c), written from the paper.

Parity status of each function (what pins it) is listed in the tests under
tests/test_oracle_*.py.
"""
