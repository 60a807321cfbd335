"""CPU oracle for tagged uniform-BLR compression.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg, never by the library.  See ``oracle.tagging``.
"""
