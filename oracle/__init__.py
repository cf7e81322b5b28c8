"""CPU oracle for Relay-BP decoding (TEST INFRASTRUCTURE ONLY).

Plain step-by-step implementations written from the paper (Sec. 2.3 and
App. A.3), used to check the CUDA decoder.  Only tests/, the package smoke
check and bench.py's CPU-baseline leg may import, call or link anything here;
the decoder library never does.
"""
