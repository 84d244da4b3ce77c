"""Binary Stereo Matching oracle: test infrastructure only (see bsm_oracle.cpp)."""
