"""CPU oracle for the dictionary-string decoder.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the decoder library
never does.  The decoder itself is plain C (``fp_oracle.c``, compiled with
gcc by :func:`build`); the greedy encoder (:mod:`oracle.encode`) is plain
Python.  Neither shares code with the CUDA path.
"""
from .core import (build, decode, decode_mt, decode_column, decode_packed, decode_rows, decoded_size,  # noqa: F401
                   sidecar, unpack12,
                   OracleResult,
                   OK, ERR_ARG, ERR_CORRUPT, ERR_CAPACITY, ERR_OVERFLOW,
                   BIT_CORRUPT, BIT_CAPACITY, BIT_OVERFLOW)
from .encode import greedy_encode, encode_column  # noqa: F401
