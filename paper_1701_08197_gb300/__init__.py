"""GB300-native LOFAR Online Flagger (LOF) hot path.

The flagger of "Towards Exascale Real-Time RFI Mitigation" (van Nieuwpoort,
2017): power from complex voltages, SumThreshold over the time-integrated
spectrum, robust pooled statistics, SumThreshold in time per channel, the
history flagger, and the flag mask applied to the data -- all in hand-written
sm_103a CUDA behind a small C ABI (include/lof.h).  This package holds the
ctypes binding (lof.py), the build step (build.py) and the seeded synthetic
workloads (synth.py).
"""
