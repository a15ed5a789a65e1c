"""FP64 CPU oracle for the Gaussian-splatting forward path.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the CUDA library or its binding.
"""
