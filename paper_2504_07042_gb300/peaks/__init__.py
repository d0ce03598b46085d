"""Pipe-throughput probes of the GPU (FP64, FP32, conversions, mma.sync, copy).

  python -m paper_2504_07042_gb300.peaks   -> compiles pipe_peaks.cu with nvcc, runs it, prints JSON
"""
