"""GB300-native (sm_103a) data-parallel BlockQuicksort."""
