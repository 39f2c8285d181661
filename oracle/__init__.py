"""FP64 CPU oracle for the ph-AFQMC walker step.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.
"""
