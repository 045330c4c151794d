"""B300-native (sm_103a) per-frame path of Akamine et al., "Fully automatic
extraction of salient objects from videos in near real-time" (arXiv:1008.0502):
saliency map -> Kalman-updated saliency prior -> MRF terms -> exact grid min cut.

Submodules (imported on demand so that the input generator works without the
CUDA library):
  seg    ctypes binding of include/seg.h (libseg.so); fails loudly if unbuilt
  synth  seeded synthetic video and graph inputs
  build  nvcc build of libseg.so
"""
__all__ = ["seg", "synth", "build"]
