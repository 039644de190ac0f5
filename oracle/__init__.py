"""CPU FP64 oracle for the FEM lead-field build — test infrastructure only.

Imported by the test suite, by the package smoke check and by the benchmark's
CPU-baseline leg; never by the product path.
"""
